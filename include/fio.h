/*
 * fio.h -- C ABI of the GB300 butterfly library for discrete Fourier integral
 * operators (Candes, Demanet & Ying, "A Fast Butterfly Algorithm for the
 * Computation of Fourier Integral Operators", 2008).
 *
 * The operator (Sec. 1, eq. dfio) is
 *     u(x) = sum_{k in Omega} e^{2 pi i Phi(x,k)} f(k),   x in X,
 * X = {(i1/N, i2/N): 0 <= i1,i2 < N}, Omega = {(k1,k2): -N/2 <= k1,k2 < N/2},
 * N a power of two.  fio_apply evaluates it with the butterfly algorithm of
 * Sec. 4 in the polar coordinates p of eq. polar (k = (sqrt2/2) N p1
 * (cos 2 pi p2, sin 2 pi p2)), with the level truncation of Sec. 5:
 *   initialization  (eq. alg2a)  pairs (A at level s, B at level L-s)
 *   recursion in p  (eq. alg2b)  levels s+1 .. floor(L/2)
 *   switch          (eq. alg2m)  at level floor(L/2)
 *   recursion in x  (eq. alg2c)  levels floor(L/2)+1 .. L-s
 *   termination     (eq. alg2d)  summing the boxes B at level s
 * fio_apply_adjoint applies the exact conjugate transpose of that discrete
 * butterfly (the steps above transposed and conjugated, in reverse order).
 *
 * Data layout (row-major, interleaved complex; complex128 for FIO_F64,
 * complex64 for FIO_F32; a torch tensor of shape (nrhs, N, N)):
 *   f, fbar : element (r, k1 + N/2, k2 + N/2) is the source of RHS r at (k1, k2)
 *   u, g    : element (r, i1, i2) is the potential of RHS r at x = (i1/N, i2/N)
 *
 * Ownership: every data pointer passed in belongs to the caller and is never
 * freed or retained past the call.  A plan owns its device tables and state
 * buffers; fio_destroy releases them.  All work of fio_apply* is enqueued on
 * the given CUDA stream (NULL = the legacy default stream) and the call returns
 * without synchronising, except where stated.
 *
 * Errors: every entry point returns FIO_OK (0) or a negative status; nothing
 * throws across the ABI.  fio_last_error() returns a thread-local message for
 * the last failing call on the calling thread.  No entry point ever falls back
 * to a CPU computation.
 */
#ifndef FIO_H_
#define FIO_H_

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct fio_plan_s *fio_plan_t;

enum {
  FIO_OK = 0,
  FIO_EINVAL = -1,   /* an argument is out of range or a pointer is NULL */
  FIO_ENOMEM = -2,   /* a device or host allocation failed */
  FIO_ECUDA = -3,    /* a CUDA runtime call failed (message has the CUDA error) */
  FIO_ETIMEOUT = -4, /* a bounded device-side wait of a tensor-core kernel expired (fio_check) */
  FIO_EDEVICE = -5   /* no usable CUDA device */
};

/* Arithmetic forms.  FIO_F64: every step in FP64.  FIO_F32: coefficients,
 * interpolation and accumulation in FP32; every phase Phi(x,k) is evaluated and
 * reduced modulo 1 in FP64 before an FP32 sin/cos; node tables in FP64. */
enum { FIO_F64 = 0, FIO_F32 = 1 };

/* Phase functions Phi(x,k), params = [a, m, b, lambda] where used:
 *   LINEAR          Phi = x.k                                   (no params)
 *   ELLIPSE         Phi = lambda x.k + sqrt(c1^2 k1^2 + c2^2 k2^2),
 *                   c1 = (a + m sin 2pi x1 sin 2pi x2)/b, c2 = (a + m cos 2pi x1 cos 2pi x2)/b
 *                   (eq. ex1 is [2, 1, 3, 1])
 *   CIRCLE          Phi = lambda x.k + c |k|, c = (a + m sin 2pi x1 sin 2pi x2)/b
 *                   (the phase of eq. ex2 is [3, 1, 4, 1])
 *   TEST_SEPARABLE  N Psi(x,p) = N (a sin 2pi x1 cos 2pi x2 + m x1 x2 + b p1 cos 2pi p2 + lambda p1^2);
 *                   its residual R^{AB} (eq. RAB) vanishes, so the butterfly is exact (tests only). */
enum { FIO_PHASE_LINEAR = 0, FIO_PHASE_ELLIPSE = 1, FIO_PHASE_CIRCLE = 2, FIO_PHASE_TEST_SEPARABLE = 3 };

/*
 * fio_plan -- build a plan for N x N grids (host work in FP64, then one upload).
 *   N         power of two, 4 <= N <= 4096
 *   q         Chebyshev points per dimension (Sec. 3.2); one of 3, 5, 7, 9, 11
 *   phase_id  FIO_PHASE_*; params/nparams: 0 (LINEAR) or 4 doubles (others)
 *   precision FIO_F64 or FIO_F32
 *   nrhs_max  largest nrhs later passed to fio_apply* (>= 1); sizes the state
 *   s         truncation depth of Sec. 5 (-1 = 3); clipped to floor(L/2)
 *   e         angular refinement of the T_P boxes: a box at level j has width
 *             2^-j in p1 and 2^-(j+e) in p2 (-1 = 2; 0 is the square-box
 *             statement of Sec. 1.1; 0 <= e <= 4)
 * For FIO_F32 it also times the switch kernels (FP32 FMA and tensor-core variants) and
 * the translation subtile widths once on its own buffers and keeps the fastest
 * (fio_plan_info().switch_impl, .trans_rs).
 * Allocates device memory on the current CUDA device; the plan may only be
 * used with that device current.  Returns FIO_EINVAL for bad arguments,
 * FIO_ENOMEM when the state does not fit, FIO_EDEVICE without a device.
 */
int fio_plan(fio_plan_t *out, int N, int q, int phase_id, const double *params, int nparams, int precision,
             int nrhs_max, int s, int e);

/* fio_destroy -- free a plan (waits for the device to finish with it). NULL is a no-op.
 * Also drops every batch that fio_apply_batch built over this plan. */
int fio_destroy(fio_plan_t plan);

/*
 * fio_workspace_bytes -- device bytes of the working state an apply with nrhs
 * right-hand sides needs: two levels of expansion coefficients (Sec. 4: only two
 * consecutive levels are ever live), 2 x 2^e N^2 pairs x nrhs x q^2 complex values.
 * The plan allocates this for nrhs_max itself (it holds its state buffers for its
 * lifetime); the figure tells a caller how much of its memory budget a plan of a
 * given size takes.  0 for a NULL plan or nrhs < 1.
 */
size_t fio_workspace_bytes(fio_plan_t plan, int nrhs);

/*
 * fio_apply -- u = B f for nrhs right-hand sides (Sec. 4, eqs. alg2a-alg2d).
 *   f, u   DEVICE pointers, layout above, complex dtype of the plan's precision;
 *          must not overlap; 16-byte aligned
 *   nrhs   1 <= nrhs <= nrhs_max
 *   stream cudaStream_t (as void*), NULL = default stream
 */
int fio_apply(fio_plan_t plan, const void *f, void *u, int nrhs, void *stream);

/* fio_apply_adjoint -- fbar = B^H g, the exact conjugate transpose of fio_apply.
 * g has u's layout, fbar has f's; DEVICE pointers; otherwise as fio_apply. */
int fio_apply_adjoint(fio_plan_t plan, const void *g, void *fbar, int nrhs, void *stream);

/*
 * fio_apply_host -- fio_apply (adjoint != 0: fio_apply_adjoint) on HOST buffers.
 * Copies the input to a plan-owned device staging buffer, applies, copies the
 * output back and synchronises the stream before returning.  Host buffers
 * should be page-locked for asynchronous copies.
 */
int fio_apply_host(fio_plan_t plan, const void *in_host, void *out_host, int nrhs, int adjoint, void *stream);

/*
 * fio_debug_stage -- run the forward butterfly on f (DEVICE, one RHS taken as
 * RHS 0 of an nrhs=1 call) up to stage j and copy that state into out (DEVICE,
 * complex128).  Stages: 0 initialization, then one per p-level, the switch, one
 * per x-level (fio_plan_info().nstages in all).  out holds the pairs (A,B) at
 * the stage's level l as [a1][a2][b1][b2][t1][t2], a in [0,2^l)^2,
 * b in [0,2^(L-l)) x [0,2^(L-l+e)), t in [0,q)^2.  Synchronises the stream.
 */
int fio_debug_stage(fio_plan_t plan, const void *f, int stage, void *out, void *stream);

typedef struct {
  int N, L, q, s, e, l0, lm, l1, phase_id, precision, nrhs_max;
  int nstages;             /* init + (lm-l0) p-levels + switch + (l1-lm) x-levels */
  long long pairs_per_level; /* 2^e N^2 */
  long long state_bytes;   /* device bytes of the two state buffers */
  long long table_bytes;   /* device bytes of the plan's tables */
  int max_box_sources;     /* most sources in one initialization box B */
  int switch_impl;         /* FIO_F32: switch kernel chosen by fio_plan's autotuner,
                              0 = FP32 FMA (one pair per CTA), 1 = tensor cores (tcgen05,
                              split TF32, kernel matrix in shared memory), 2 = FP32 FMA,
                              warp-specialised and persistent, 3 = tensor cores with the
                              kernel matrix in tensor memory (persistent, one CTA per SM),
                              4 = as 3 with the split-TF32 products as two wide MMAs per
                              K-step (N = 192 and N = 128), 5 and 6 = as 3 and 4 with three
                              split-TF32 products (A0 B0 + A0 B1 + A1 B0, each entry within
                              ~3 * 2^-22 of |A||B|) instead of five */
  int trans_rs;            /* FIO_F32, translations of the p-shape (recursion in p, eq. alg2b, and
                              the adjoint of the recursion in x): right-hand sides per subtile
                              (2, 4 or 8), or 32 for the register-tiled kernel (one RHS per lane,
                              q <= 9); chosen by fio_plan's autotuner */
  int switch_rhs_tile;     /* FIO_F32, switch kernels 0 and 2: right-hand sides per contraction
                              task (4 or 8), chosen by fio_plan's autotuner */
  int trans_rs_x;          /* FIO_F32, translations of the x-shape (recursion in x, eq. alg2c, and
                              the adjoint of the recursion in p): 2, 4 or 8, or 32 (register-tiled) */
} fio_plan_info_t;

/* fio_plan_info -- copy the plan's parameters and sizes into *info. */
int fio_plan_info(fio_plan_t plan, fio_plan_info_t *info);

/* fio_check -- synchronise the stream and report device-side failures of earlier
 * applies with this plan: FIO_ETIMEOUT if a kernel's bounded wait on the tensor
 * cores expired (that apply's output is invalid; the flag is then cleared),
 * FIO_OK otherwise.  fio_apply_host calls it itself. */
int fio_check(fio_plan_t plan, void *stream);

/* fio_plan_set_wait_limit -- for tests of the failure path: the limit, in ns, of the
 * waits by which the tensor-memory switch kernels (switch_impl 3-6) hand chunks between
 * its producer warps and its MMA warp (0 restores the normal 2 s).  A tiny limit makes
 * those waits expire: the kernel then records the expiry, stops issuing work, still waits
 * with the normal limit for the tensor-core operations it issued, frees its tensor memory
 * and returns; fio_check reports FIO_ETIMEOUT and the output of that apply is invalid.
 * The paper has no counterpart. */
int fio_plan_set_wait_limit(fio_plan_t plan, unsigned long long ns);

/* fio_plan_set_switch -- override the autotuner's choice of the FIO_F32 switch
 * kernel: impl 0 = FP32 FMA, 1 = tensor cores (kernel matrix in shared memory),
 * 2 = warp-specialised FP32 FMA, 3 = tensor cores (kernel matrix in tensor memory), 4 = as 3
 * with two wide MMAs per K-step, 5 and 6 = as 3 and 4 with three split-TF32 products.
 * FIO_EINVAL if the plan is FIO_F64 or the kernel does not fit this plan (its
 * shared memory need: 1 and 2 are not available for every q). */
int fio_plan_set_switch(fio_plan_t plan, int impl);

/* fio_plan_set_tuning -- override every choice of fio_plan's autotuner for an FIO_F32
 * plan (a value of -1 keeps the current choice): switch_impl as fio_plan_set_switch,
 * switch_rhs_tile 4 or 8 (kernel 0 only; kernel 2 uses 4); the translation kernels of
 * each shape: trans_rs (p-shape) and trans_rs_x (x-shape), 2, 4 or 8 (RHS subtiles) or
 * 32 (register-tiled kernels, q <= 9).
 * FIO_EINVAL for FIO_F64 plans or values outside those sets. */
int fio_plan_set_tuning(fio_plan_t plan, int switch_impl, int switch_rhs_tile, int trans_rs, int trans_rs_x);

/*
 * fio_apply_amplitude -- an FIO with a variable amplitude (eq. allfio),
 *     u(x) = sum_k a(x,k) e^{2 pi i Phi(x,k)} f(k),  a(x,k) = sum_{t < nt} g_t(x) h_t(k),
 * the separated form the paper gives for it: the nt products f_t = h_t f are the
 * right-hand sides of ONE butterfly apply, so every phase evaluation is shared by all of
 * them (the "vectorised" butterfly), then u = sum_t g_t (B f_t), summed over t in order.
 * adjoint != 0 applies the conjugate transpose: fbar(k) = sum_x conj a(x,k)
 * e^{-2 pi i Phi(x,k)} gin(x) = sum_t conj h_t(k) (B^H (conj g_t gin))(k).
 *   in, out  DEVICE (nrhs, N, N) in the plan's complex dtype (f and u; gin and fbar)
 *   g        DEVICE (nt, N, N): g_t on X, element (t, i1, i2)
 *   h        DEVICE (nt, N, N): h_t on Omega, element (t, k1 + N/2, k2 + N/2)
 *   nt, nrhs nt * nrhs <= nrhs_max
 * Uses the plan's two staging buffers (allocated on first use, nrhs_max N^2 elements
 * each): one call at a time per plan.
 */
int fio_apply_amplitude(fio_plan_t plan, const void *in, const void *g, const void *h, int nt, void *out, int nrhs,
                        int adjoint, void *stream);

/*
 * fio_apply_wave -- a sum of two FIOs on the same input (Sec. 1: the solution operator of
 * the wave equation u_tt = c^2 Lap u with u_t(x, 0) = 0 is
 *     u(x, t) = 1/2 sum_k (e^{2 pi i (x.k + c|k|t)} + e^{2 pi i (x.k - c|k|t)}) f(k),
 * f the Fourier coefficients of u(x, 0); with FIO_PHASE_CIRCLE plans of params
 * [+a t, +m t, b, 1] and [-a t, -m t, b, 1] this is that pair, with the speed
 * c(x) = (a + m sin 2 pi x1 sin 2 pi x2)/b):
 *     out = w_plus B_plus in + w_minus B_minus in          (adjoint == 0)
 *     out = w_plus B_plus^H in + w_minus B_minus^H in      (adjoint != 0)
 *   plus, minus  plans of the same N, precision and device (any phases)
 *   in, out      DEVICE (nrhs, N, N) in the plans' complex dtype, different buffers
 *   nrhs         1 <= nrhs <= both plans' nrhs_max
 * B_minus's result goes through the minus plan's first staging buffer (allocated on first
 * use): one call at a time per plan.  Enqueued on `stream`.
 */
int fio_apply_wave(fio_plan_t plus, fio_plan_t minus, const void *in, void *out, int nrhs, double w_plus,
                   double w_minus, int adjoint, void *stream);

/*
 * fio_apply_wave_series -- the wave propagator at several times from ONE plan (Sec. 1):
 *     out[k] = 1/2 (B_{+t_k} in + B_{-t_k} in),   k = 0 .. ntimes-1,
 * where B_{+-t} has the phase lambda x.k +- t c(x)|k|, c(x) = (a + m sin 2 pi x1 sin 2 pi x2)/b,
 * and plan is a FIO_PHASE_CIRCLE plan with params [a, m, b, lambda] (the speed at t = 1).
 * With lambda = 1 and in the Fourier coefficients of u(x, 0), out[k] is u(x, t_k) for
 * u_tt = c^2 Lap u, u_t(x, 0) = 0 (exactly for constant c).  Every one of the 2 ntimes
 * butterflies runs on this plan's node, source and Lagrange tables and its two state
 * buffers -- the tables do not depend on the phase, only the kernels' phase arguments
 * change -- so the series needs one plan's device memory (fio_plan_info().table_bytes +
 * state_bytes, plus one staging buffer of nrhs_max N^2 elements allocated on first use)
 * instead of 2 ntimes plans'.  Each out[k] is bit-identical to fio_apply_wave on a
 * separately built pair of plans with params [+-a t_k, +-m t_k, b, lambda].
 *   times  HOST, ntimes values
 *   in     DEVICE (nrhs, N, N); out DEVICE (ntimes, nrhs, N, N); not overlapping
 * Enqueued on `stream`; uses the plan's state: one call at a time per plan.
 */
int fio_apply_wave_series(fio_plan_t plan, const double *times, int ntimes, const void *in, void *out, int nrhs,
                          void *stream);

/*
 * fio_direct -- the operator itself (eq. dfio), summed directly on the GPU at sampled
 * grid points: out[r][i] = sum_k e^{2 pi i Phi(x_i,k)} f[r](k), x_i = the flat grid index
 * xi[i] = i1 * N + i2.  Every term of the N^2 is evaluated (O(N^2) per point), the phase as
 * the plan's butterfly does (double-float for FIO_F32, FP64 for FIO_F64) and the sum
 * accumulated in FP64 in a fixed order.  The reference against which the error of
 * eq. err is estimated.
 *   f    DEVICE, (nrhs, N, N) in the plan's complex dtype; 1 <= nrhs <= 65535
 *   xi   DEVICE, nx int64 flat indices in [0, N^2) (not checked on the device)
 *   out  DEVICE, (nrhs, nx) complex128
 * Enqueued on `stream`; does not synchronise.
 */
int fio_direct(fio_plan_t plan, const void *f, int nrhs, const long long *xi, int nx, void *out, void *stream);

/*
 * fio_plan_auto -- a plan whose q meets a target accuracy (Sec. 5: the error falls
 * geometrically with q, so the paper's recipe is to raise q until eq. err is small
 * enough).  For q = 3, 5, 7, 9, 11 in turn it builds the plan (arguments as fio_plan),
 * applies it to a seeded complex white-noise input and estimates the relative L2 error of
 * eq. err on nsample seeded grid points against fio_direct; it stops at the first q whose
 * estimate is <= target.  *out receives that plan (or the q = 11 plan if none meets the
 * target: then fio_last_error() says so), *q_out its q and *err_out the estimate.
 * Synchronises the device; allocates and frees scratch for one input and one output.
 */
int fio_plan_auto(fio_plan_t *out, int N, int phase_id, const double *params, int nparams, int precision, int nrhs_max,
                  int s, int e, double target, int nsample, unsigned long long seed, int *q_out, double *err_out);

/* fio_kernel_launches -- number of kernels one fio_apply (adjoint != 0: fio_apply_adjoint)
 * with nrhs right-hand sides enqueues. */
int fio_kernel_launches(fio_plan_t plan, int nrhs, int adjoint);

/* Per-kernel timing.  fio_profile(plan, 1) clears the counters and starts
 * recording a CUDA event pair on the launch stream around every kernel that
 * fio_apply* enqueues with this plan (at most 4096 launches); fio_profile(plan, 0)
 * stops.  fio_profile_read synchronises on the recorded events and fills up to
 * max entries {name, launches, total ms} for the kernel kinds that ran, setting
 * *n to their number.  Kinds: init, trans_p (eq. alg2b), switch (eq. alg2m),
 * trans_x (eq. alg2c), term (eq. alg2d) and their conjugate transposes *_adj. */
typedef struct {
  char name[24];
  long long launches;
  double ms;
} fio_kernel_time_t;
int fio_profile(fio_plan_t plan, int enable);
int fio_profile_read(fio_plan_t plan, fio_kernel_time_t *out, int max, int *n);

/* fio_peak_probe -- measure a per-GPU arithmetic peak on the current device:
 * kind 0 FP32 FMA, 1 FP64 FMA (returned as flop/s, 2 per FMA), 2 FP32 sin/cos
 * through the special-function unit (results/s).  A fixed dependent-chain
 * kernel over every SM, timed with CUDA events; synchronises the device.
 * kinds 3..8: the tensor-core rate (flop/s, 2 per multiply-add) of tcgen05.mma, M = 128,
 * one CTA per SM issuing back to back with the operands rotating over 16 K-steps:
 * A in tensor memory: 3 TF32 N = 64, 4 BF16 N = 64, 5 TF32 N = 256, 6 BF16 N = 256;
 * A in shared memory: 7 TF32 N = 64, 8 BF16 N = 64; A in tensor memory with the MMAs taking
 * 3 (kind 9) or 2 (kind 10) accumulators in turn: TF32 N = 64.
 * The paper has no counterpart: it is a measurement aid for the roofline. */
int fio_peak_probe(int kind, double *per_second);

/*
 * fio_apply_noalloc -- u = B f for small grids, allocating nothing.
 * The paper has no counterpart: this is a calling convenience.  It is for
 * callers that cannot allocate device memory when they apply the operator (an
 * embedding runtime that owns the allocator and forbids cudaMalloc after
 * start-up, a real-time loop that must not block on allocation, a plugin
 * without a memory pool): it needs no plan and calls no cudaMalloc, cudaFree or
 * allocating library routine.
 *   N, q, phase_id, params, nparams, precision, s, e: as fio_plan, with
 *          4 <= N <= 32, q in {3, 5, 7, 9}, 0 <= e <= 2
 *   f, u   DEVICE pointers as in fio_apply; nrhs >= 1
 * Its working memory -- the node and source tables and the two level buffers
 * of expansion coefficients -- lives in one static device array of 8 MiB that
 * every GPU loading this library holds until the process exits.  A problem
 * whose tables plus two levels of 2^e N^2 q^2 nrhs complex coefficients exceed
 * 8 MiB is rejected with FIO_EINVAL and a message naming both sizes.
 * The first call on a device looks up the array's device address with that
 * device current.  All calls share the array, which keeps the last call's
 * contents (every coefficient is written before it is read, so nothing needs
 * clearing): calls that overlap on the GPU (other streams, other host threads'
 * streams) race and must be serialised by the caller.  The host side copies its
 * tables from one static pageable image that the next call rebuilds, which waits
 * for earlier work on the stream; for the same reason a call on a stream that is
 * being captured returns FIO_EINVAL.  FIO_F32 runs the generic FP32 kernels (no
 * double-float phase tables), so its results agree with fio_apply's FP32 plans
 * within the FP32 tolerance, not bit for bit.
 */
int fio_apply_noalloc(int N, int q, int phase_id, const double *params, int nparams, int precision, int s, int e,
                      const void *f, void *u, int nrhs, void *stream);

/*
 * Batches of plans.  A batch applies many FIO_F32 plans -- of different N,
 * phases, right-hand-side counts and q -- as one unit: every butterfly step
 * (initialization, each level of the recursions in p and x, the switch, the
 * termination; Sec. 4) becomes ONE persistent kernel launch over the pairs of
 * all plans of a q that take that step, and the whole schedule is captured once
 * in a CUDA graph (one graph for fio_apply, one for fio_apply_adjoint).  Plans
 * of different q (or s) form separate groups whose launch chains run on
 * parallel branches of the graph.  Each plan's results are bit-identical to
 * fio_apply / fio_apply_adjoint on that plan alone with the FP32 FMA switch
 * (switch_impl 0) and the RHS-subtile translations (trans_rs, trans_rs_x 2, 4 or 8):
 * the batch uses neither the tensor-core switch nor the register-tiled translations.
 *
 * Data: one packed DEVICE buffer for all inputs and one for all outputs.  Plan i
 * occupies elements [off[i], off[i+1]) of both (complex64), laid out as
 * fio_apply's (nrhs[i], N_i, N_i) arrays; off[0] = 0 and
 * off[i+1] = off[i] + nrhs[i] N_i^2 (fio_batch_offsets).
 *
 * Ownership: the batch keeps pointers to the plans' tables and state buffers,
 * so the plans must outlive it, and none of them may be applied (alone or in
 * another batch) while an apply of this batch may be running.  One apply of a
 * batch at a time: applies on different streams race on the plans' states.
 */
typedef struct fio_batch_s *fio_batch_t;

enum {
  FIO_BATCH_TUNE = 1,  /* time each launch at several persistent grid sizes and the
                          graph with parallel and with serial groups; keep the fastest */
  FIO_BATCH_SERIAL = 2 /* capture the groups one after another (no parallel branches) */
};

/*
 * fio_batch_create -- build the schedule and the two graphs of a batch.
 *   plans   nplans distinct FIO_F32 plans (1 <= nplans <= 4096) built on the current device,
 *           each with 2^s <= 8
 *   nrhs    nplans right-hand-side counts, 1 <= nrhs[i] <= that plan's nrhs_max
 *   flags   0, FIO_BATCH_TUNE (runs every kernel a few times on scratch
 *           buffers it allocates and frees; synchronises the device) and/or
 *           FIO_BATCH_SERIAL (then tuning keeps the groups serial)
 * Without FIO_BATCH_TUNE each launch uses one CTA per resident slot of every SM
 * (occupancy x SM count, at most the launch's work) and the groups run on
 * parallel graph branches.  Allocates a small device descriptor buffer.
 */
int fio_batch_create(fio_batch_t *out, int nplans, const fio_plan_t *plans, const int *nrhs, int flags);

/*
 * fio_apply_batch -- u[i] = B_i f[i] for the nplans plans in one go, each with its own
 * DEVICE input and output pointer (layout and dtype as fio_apply; complex64; 16-byte
 * aligned; nrhs[i] right-hand sides, 1 <= nrhs[i] <= plan i's nrhs_max).
 * fio_apply_batch_adjoint -- fbar[i] = B_i^H g[i] likewise.
 * The first call for a given list of plans and nrhs builds a batch exactly as
 * fio_batch_create(plans, nrhs, 0) does and keeps it (at most 8 such batches; the
 * oldest is dropped, which synchronises the device); later calls with the same plans
 * and counts reuse it: one small kernel records the nplans pointer pairs, then one
 * graph launch runs every step, one persistent launch per step and q-group.  Results
 * are bit-identical to fio_batch_apply on packed copies of the same data.  Same rules
 * as fio_batch_apply: FIO_F32 plans only, one call at a time per set of plans, and
 * fio_destroy of any of the plans drops the kept batch.  Enqueued on `stream`.
 */
int fio_apply_batch(fio_plan_t *plans, int nplans, const void *const *f, void *const *u, const int *nrhs,
                    void *stream);
int fio_apply_batch_adjoint(fio_plan_t *plans, int nplans, const void *const *g, void *const *fbar, const int *nrhs,
                            void *stream);

/* fio_batch_destroy -- free the batch (waits for the device). NULL is a no-op. */
int fio_batch_destroy(fio_batch_t batch);

/* fio_batch_offsets -- write the nplans + 1 element offsets off[] of the packed buffers. */
int fio_batch_offsets(fio_batch_t batch, long long *off);

/*
 * fio_batch_apply -- apply every plan of the batch (adjoint != 0: its conjugate
 * transpose) to its slice of `in`, writing its slice of `out`.  in, out: DEVICE
 * pointers to packed complex64 buffers of fio_batch_offsets()[nplans] elements,
 * 16-byte aligned, not overlapping.  Enqueues one one-thread kernel (which
 * records in/out for the graph) and one graph launch on `stream`.
 */
int fio_batch_apply(fio_batch_t batch, const void *in, void *out, int adjoint, void *stream);

typedef struct {
  int nplans;
  int ngroups;           /* distinct (q, s) */
  int launches_fwd;      /* batched kernel launches in the forward graph (plus one io kernel per apply) */
  int launches_adj;      /* the same for the adjoint graph */
  int parallel_groups;   /* 1: groups on parallel graph branches, 0: one after another */
  int tuned;             /* FIO_BATCH_TUNE was given */
  long long total_elems; /* off[nplans] */
  double tune_ms;        /* host time spent autotuning */
} fio_batch_info_t;
int fio_batch_info(fio_batch_t batch, fio_batch_info_t *info);

/* fio_batch_profile -- run the batch once WITHOUT the graph, with a CUDA event
 * pair around each launch, synchronise, and fill up to max entries {name,
 * launches, total ms} per kernel kind ("b_init", "b_trans_p", ...), setting *n. */
int fio_batch_profile(fio_batch_t batch, const void *in, void *out, int adjoint, void *stream, fio_kernel_time_t *times,
                      int max, int *n);

/* fio_last_error -- thread-local message of the last failing call ("" if none). */
const char *fio_last_error(void);

/* fio_version -- library version number. */
int fio_version(void);

#ifdef __cplusplus
}
#endif

#endif /* FIO_H_ */
