// fio_noalloc.cu -- fio_apply_noalloc: the forward butterfly for small grids
// without any memory allocation.
//
// Some callers cannot allocate device memory when they need an apply: code
// whose allocator is owned by someone else (an embedding runtime that forbids
// cudaMalloc after start-up, a real-time loop that must not block on the
// allocator, a plugin without its own memory pool).  For them this entry point
// keeps everything the butterfly needs besides the caller's f and u -- the node
// and source tables and the two level buffers of expansion coefficients -- in
// one file-scope device array of fixed size, and builds the host side of the
// tables in fixed-size static host buffers.  It calls no cudaMalloc, cudaFree
// or allocating library routine.  The level schedule is fio_apply's; the FP32
// form runs the generic FP32 kernels (no double-float phase tables are built
// here), which agree with fio_apply's FP32 plans within the FP32 tolerance, not
// bit for bit.  The tables are copied from one static host image that the next
// call rebuilds, so a call on a stream that is being captured is refused: a
// replayed copy would read whatever the image holds at replay time.
#include <cuda_runtime.h>

#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <mutex>

#include "fio.h"
#include "fio_run.cuh"

namespace fio {
void set_last_error(const char *msg);
int run_q3(const PlanDev &, int, const void *, void *, int, cudaStream_t, int, int *);
int run_q5(const PlanDev &, int, const void *, void *, int, cudaStream_t, int, int *);
int run_q7(const PlanDev &, int, const void *, void *, int, cudaStream_t, int, int *);
int run_q9(const PlanDev &, int, const void *, void *, int, cudaStream_t, int, int *);
}  // namespace fio

namespace {

using namespace fio;

// The shared scratch: every device that loads the library holds these 8 MiB
// until the process exits.
constexpr size_t kScratchBytes = (size_t)8 << 20;
static __device__ __align__(256) unsigned char g_scratch[kScratchBytes];

constexpr int kMaxN = 32, kMaxE = 2, kMaxDevices = 64;
constexpr int kMaxNN = kMaxN * kMaxN;
constexpr int kMaxBoxes = kMaxN * (kMaxN << kMaxE);                    // T_P boxes at level L-s

// Host-side table images (no heap): built, then copied into g_scratch.
static unsigned char g_host[1 << 20];
static long long g_boxof[kMaxNN];
static double g_p1[kMaxNN], g_p2[kMaxNN];
static int g_cnt[kMaxBoxes + 1], g_pos[kMaxBoxes];

static void *g_dev_ptr[kMaxDevices];  // device address of g_scratch, per device
static std::mutex g_mu;               // serialises the host side of concurrent calls

int fail(int code, const char *fmt, ...) {
  char msg[256];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(msg, sizeof msg, fmt, ap);
  va_end(ap);
  set_last_error(msg);
  return code;
}

const double kTwoPi = 6.283185307179586476925286766559;

void cheb_grid(int q, double *z) {
  for (int j = 0; j < q; j++) z[j] = 0.5 * std::sin(M_PI * (q - 1 - 2 * j) / (2.0 * (q - 1)));
}

void lagrange_all(int q, const double *z, double t, double *out) {
  double den = 0.0;
  for (int j = 0; j < q; j++)
    if (t == z[j]) {
      for (int i = 0; i < q; i++) out[i] = i == j ? 1.0 : 0.0;
      return;
    }
  for (int j = 0; j < q; j++) {
    double w = (j & 1) ? -1.0 : 1.0;
    if (j == 0 || j == q - 1) w *= 0.5;
    out[j] = w / (t - z[j]);
    den += out[j];
  }
  for (int j = 0; j < q; j++) out[j] /= den;
}

size_t al256(size_t x) { return (x + 255) & ~(size_t)255; }

}  // namespace

extern "C" int fio_apply_noalloc(int N, int q, int phase_id, const double *params, int nparams, int precision,
                                 int s, int e, const void *f, void *u, int nrhs, void *stream) {
  int L = 0;
  while ((1 << L) < N && L < 30) L++;
  if (N < 4 || N > kMaxN || (1 << L) != N) return fail(FIO_EINVAL, "N=%d must be a power of two in [4, %d]", N, kMaxN);
  if (q != 3 && q != 5 && q != 7 && q != 9) return fail(FIO_EINVAL, "q=%d must be 3, 5, 7 or 9", q);
  if (phase_id < 0 || phase_id > 3) return fail(FIO_EINVAL, "unknown phase_id %d", phase_id);
  if (phase_id != FIO_PHASE_LINEAR && (nparams != 4 || !params))
    return fail(FIO_EINVAL, "phase %d needs 4 params, got %d", phase_id, nparams);
  if ((phase_id == FIO_PHASE_ELLIPSE || phase_id == FIO_PHASE_CIRCLE) && params[2] == 0.0)
    return fail(FIO_EINVAL, "params[2] (b) must be nonzero");
  if (precision != FIO_F64 && precision != FIO_F32) return fail(FIO_EINVAL, "unknown precision %d", precision);
  if (s < 0) s = 3;
  if (s > L / 2) s = L / 2;
  if (e < 0) e = 2;
  if (e > kMaxE) return fail(FIO_EINVAL, "e=%d must be in [0, %d]", e, kMaxE);
  if (nrhs < 1) return fail(FIO_EINVAL, "nrhs=%d must be >= 1", nrhs);
  if (!f || !u) return fail(FIO_EINVAL, "NULL data pointer");
  if (((uintptr_t)f | (uintptr_t)u) & 15) return fail(FIO_EINVAL, "data pointers must be 16-byte aligned");
  cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
  if (cudaStreamIsCapturing((cudaStream_t)stream, &cap) != cudaSuccess || cap != cudaStreamCaptureStatusNone)
    return fail(FIO_EINVAL, "fio_apply_noalloc cannot run while its stream is being captured: it copies its tables "
                            "from a host image that the next call rewrites");

  const long long NN = (long long)N * N;
  const int lb = L - s;
  const long long nb1 = 1LL << lb, nb2 = 1LL << (lb + e), nbox = nb1 * nb2;
  int nx = 0, np2 = 0;
  for (int l = 0; l <= L; l++) {
    nx += (1 << l) * (q + 1);
    np2 += (1 << (l + e)) * (q + 1);
  }
  const size_t b_x = al256(nx * sizeof(XNode)), b_p1 = al256(nx * sizeof(P1Node)), b_p2 = al256(np2 * sizeof(P2Node)),
               b_g = al256(N * sizeof(XNode)), b_s = al256(NN * sizeof(Src)), b_f = al256(NN * sizeof(int)),
               b_w = al256(NN * 2 * q * sizeof(double)), b_o = al256((nbox + 1) * sizeof(int));
  const size_t tbytes = b_x + b_p1 + b_p2 + b_g + b_s + b_f + b_w + b_o;
  const size_t sbytes = al256((((size_t)NN * q * q) << e) * (size_t)nrhs * (precision == FIO_F64 ? 16 : 8));
  if (tbytes > sizeof g_host || tbytes + 2 * sbytes > kScratchBytes)
    return fail(FIO_EINVAL, "this problem needs %zu bytes of scratch; the static limit is %zu bytes", tbytes + 2 * sbytes,
                kScratchBytes);

  std::lock_guard<std::mutex> lock(g_mu);
  int dev = 0;
  cudaError_t ce = cudaGetDevice(&dev);
  if (ce != cudaSuccess) return fail(FIO_EDEVICE, "no CUDA device: %s", cudaGetErrorString(ce));
  if (dev < 0 || dev >= kMaxDevices) return fail(FIO_EDEVICE, "device %d beyond %d", dev, kMaxDevices);
  if (!g_dev_ptr[dev]) {  // once per device, with that device current
    void *ptr = nullptr;
    ce = cudaGetSymbolAddress(&ptr, g_scratch);
    if (ce != cudaSuccess || !ptr) return fail(FIO_ECUDA, "cudaGetSymbolAddress: %s", cudaGetErrorString(ce));
    g_dev_ptr[dev] = ptr;
  }
  char *dbase = (char *)g_dev_ptr[dev];

  PlanDev d;
  memset(&d, 0, sizeof d);
  d.N = N;
  d.L = L;
  d.q = q;
  d.s = s;
  d.e = e;
  d.l0 = s;
  d.lm = L / 2;
  d.l1 = L - s;
  d.precision = precision;
  d.nrhs_max = nrhs;
  cudaDeviceGetAttribute(&d.smem_optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
  d.ph.id = phase_id;
  d.ph.N = N;
  if (phase_id == FIO_PHASE_ELLIPSE || phase_id == FIO_PHASE_CIRCLE) {
    d.ph.a = params[0];
    d.ph.m = params[1];
    d.ph.ib = 1.0 / params[2];
    d.ph.lam = params[3];
  } else if (phase_id == FIO_PHASE_TEST_SEPARABLE) {
    d.ph.sa = params[0];
    d.ph.sm = params[1];
    d.ph.sb = params[2];
    d.ph.sl = params[3];
  }
  double z[kQMax], lg[kQMax];
  cheb_grid(q, z);
  for (int sg = 0; sg < 2; sg++)
    for (int jp = 0; jp < q; jp++) {
      lagrange_all(q, z, (2 * sg - 1) / 4.0 + 0.5 * z[jp], lg);
      for (int j = 0; j < q; j++) d.T[sg][j][jp] = lg[j];
    }
  const int M = 1 << s;
  for (int m = 0; m < M; m++) {
    lagrange_all(q, z, (double)m / M - 0.5, lg);
    for (int j = 0; j < q; j++) d.V[m][j] = lg[j];
  }

  // host images of the tables, in the order they sit in the scratch
  memset(g_host, 0, tbytes);
  XNode *xnode = (XNode *)g_host;
  P1Node *p1node = (P1Node *)(g_host + b_x);
  P2Node *p2node = (P2Node *)(g_host + b_x + b_p1);
  XNode *xgrid = (XNode *)(g_host + b_x + b_p1 + b_p2);
  Src *src = (Src *)(g_host + b_x + b_p1 + b_p2 + b_g);
  int *srcf = (int *)(g_host + b_x + b_p1 + b_p2 + b_g + b_s);
  double *srcw = (double *)(g_host + b_x + b_p1 + b_p2 + b_g + b_s + b_f);
  int *boxoff = (int *)(g_host + b_x + b_p1 + b_p2 + b_g + b_s + b_f + b_w);
  int ix = 0, i2 = 0;
  for (int l = 0; l <= L; l++) {
    d.tb.xoff[l] = d.tb.p1off[l] = ix;
    d.tb.p2off[l] = i2;
    const double w = 1.0 / (double)(1 << l);
    for (int a = 0; a < (1 << l); a++)
      for (int j = 0; j <= q; j++, ix++) {
        xnode[ix].x = (a + 0.5 + (j < q ? z[j] : 0.0)) * w;
        xnode[ix].s = std::sin(kTwoPi * xnode[ix].x);
        xnode[ix].c = std::cos(kTwoPi * xnode[ix].x);
        p1node[ix].p1 = xnode[ix].x;
        p1node[ix].rho = 0.5 * std::sqrt(2.0) * N * p1node[ix].p1;
      }
    const double w2 = 1.0 / (double)(1LL << (l + e));
    for (long long b = 0; b < (1LL << (l + e)); b++)
      for (int j = 0; j <= q; j++, i2++) {
        const double p2 = (b + 0.5 + (j < q ? z[j] : 0.0)) * w2;
        p2node[i2].c = std::cos(kTwoPi * p2);
        p2node[i2].s = std::sin(kTwoPi * p2);
      }
  }
  for (int i = 0; i < N; i++) {
    xgrid[i].x = (double)i / N;
    xgrid[i].s = std::sin(kTwoPi * xgrid[i].x);
    xgrid[i].c = std::cos(kTwoPi * xgrid[i].x);
  }
  for (long long b = 0; b <= nbox; b++) g_cnt[b] = 0;
  for (long long kf = 0; kf < NN; kf++) {
    const int k1 = (int)(kf / N) - N / 2, k2 = (int)(kf % N) - N / 2;
    const double kk = (double)k1 * k1 + (double)k2 * k2;
    const double p1 = std::sqrt(2.0 * kk) / N;
    double ang = std::atan2((double)k2, (double)k1) / kTwoPi;
    if (ang < 0.0) ang += 1.0;
    if (k1 == 0 && k2 == 0) ang = 0.0;
    long long b1 = (long long)std::floor(p1 * (double)nb1);
    long long b2 = (long long)std::floor(ang * (double)nb2);
    if (b1 > nb1 - 1) b1 = nb1 - 1;
    if (b2 > nb2 - 1) b2 = nb2 - 1;
    g_boxof[kf] = b1 * nb2 + b2;
    g_p1[kf] = p1;
    g_p2[kf] = ang;
    g_cnt[g_boxof[kf] + 1]++;
  }
  int maxsrc = 0;
  for (long long b = 0; b < nbox; b++) {
    maxsrc = std::max(maxsrc, g_cnt[b + 1]);
    g_cnt[b + 1] += g_cnt[b];
  }
  for (long long b = 0; b < nbox; b++) {
    g_pos[b] = g_cnt[b];
    boxoff[b] = g_cnt[b];
  }
  boxoff[nbox] = g_cnt[nbox];
  for (long long kf = 0; kf < NN; kf++) {
    const int j = g_pos[g_boxof[kf]]++;
    const int k1 = (int)(kf / N) - N / 2, k2 = (int)(kf % N) - N / 2;
    src[j].k1 = k1;
    src[j].k2 = k2;
    src[j].kr = std::sqrt((double)k1 * k1 + (double)k2 * k2);
    src[j].p1 = g_p1[kf];
    src[j].c2 = std::cos(kTwoPi * g_p2[kf]);
    srcf[j] = (int)kf;
    const long long b1 = g_boxof[kf] / nb2, b2 = g_boxof[kf] % nb2;
    lagrange_all(q, z, g_p1[kf] * (double)nb1 - (double)b1 - 0.5, &srcw[(size_t)j * 2 * q]);
    lagrange_all(q, z, g_p2[kf] * (double)nb2 - (double)b2 - 0.5, &srcw[(size_t)j * 2 * q + q]);
  }
  d.maxsrc = maxsrc;
  d.nbox_init = (int)nbox;
  d.tb.xnode = (const XNode *)dbase;
  d.tb.p1node = (const P1Node *)(dbase + b_x);
  d.tb.p2node = (const P2Node *)(dbase + b_x + b_p1);
  d.tb.xgrid = (const XNode *)(dbase + b_x + b_p1 + b_p2);
  d.tb.src = (const Src *)(dbase + b_x + b_p1 + b_p2 + b_g);
  d.tb.src_f = (const int *)(dbase + b_x + b_p1 + b_p2 + b_g + b_s);
  d.tb.src_w = (const double *)(dbase + b_x + b_p1 + b_p2 + b_g + b_s + b_f);
  d.tb.box_off = (const int *)(dbase + b_x + b_p1 + b_p2 + b_g + b_s + b_f + b_w);
  d.state[0] = dbase + tbytes;
  d.state[1] = dbase + tbytes + sbytes;
  d.prof = nullptr;

  // The copy from this pageable host image returns once the image has been
  // staged, so the next call may rebuild it; the kernels below run after it
  // on the same stream.  Every state element is written before it is read, so
  // the level buffers need no clearing between calls.
  cudaStream_t st = (cudaStream_t)stream;
  if ((ce = cudaMemcpyAsync(dbase, g_host, tbytes, cudaMemcpyHostToDevice, st)) != cudaSuccess)
    return fail(FIO_ECUDA, "cudaMemcpyAsync(tables): %s", cudaGetErrorString(ce));
  int rc = 0;
  switch (q) {
  case 3: rc = run_q3(d, RUN_FWD, f, u, nrhs, st, -1, nullptr); break;
  case 5: rc = run_q5(d, RUN_FWD, f, u, nrhs, st, -1, nullptr); break;
  case 7: rc = run_q7(d, RUN_FWD, f, u, nrhs, st, -1, nullptr); break;
  case 9: rc = run_q9(d, RUN_FWD, f, u, nrhs, st, -1, nullptr); break;
  }
  if (rc) return fail(FIO_ECUDA, "fio_apply_noalloc: %s", cudaGetErrorString((cudaError_t)rc));
  return FIO_OK;
}
