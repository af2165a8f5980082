// fio_plan.cu -- plan construction (host, FP64) and the C ABI of include/fio.h.
//
// A plan holds, on the device, every table the kernels read:
//   * node coordinates of the boxes of T_X and T_P at every level (Sec. 3.2
//     Chebyshev grid adapted to a box: centre + width * z_j), with sin/cos of
//     the x coordinates and the polar factors (sqrt2/2) N p1, cos/sin 2 pi p2 of
//     the p coordinates (Sec. 1.1, eq. polar);
//   * the sources k of Omega sorted by their box B at level L - s, with the two
//     1D Lagrange weight vectors L_j(phat) of each (eq. alg2a);
//   * two state buffers (only two consecutive levels are ever live, Sec. 4).
// The 1D translation matrices T^0, T^1 and the termination matrix V are
// position- and level-independent (Sec. 4) and travel as kernel arguments.
#include <atomic>
#include <cuda_runtime.h>

#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <new>
#include <string>
#include <vector>

#include "fio.h"
#include "fio_internal.cuh"



namespace {

thread_local std::string g_err;

int fail(int code, const char *fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof buf, fmt, ap);
  va_end(ap);
  g_err = buf;
  return code;
}

int cuda_fail(cudaError_t e, const char *what) {
  return fail(e == cudaErrorMemoryAllocation ? FIO_ENOMEM : FIO_ECUDA, "%s: %s", what, cudaGetErrorString(e));
}

const double kTwoPi = 6.283185307179586476925286766559;

// Chebyshev grid of order q on [-1/2, 1/2], z_j = cos(j pi/(q-1))/2, written in
// the sine form sin(pi (q-1-2j) / (2(q-1)))/2, which is exactly antisymmetric.
void cheb_grid(int q, double *z) {
  for (int j = 0; j < q; j++) z[j] = 0.5 * std::sin(M_PI * (q - 1 - 2 * j) / (2.0 * (q - 1)));
}

// All q Lagrange polynomials of the grid at t, barycentric form (second kind)
// with the Chebyshev-Lobatto weights (-1)^j, halved at both ends.
void lagrange_all(int q, const double *z, double t, double *out) {
  double den = 0.0;
  for (int j = 0; j < q; j++) {
    if (t == z[j]) {
      for (int i = 0; i < q; i++) out[i] = i == j ? 1.0 : 0.0;
      return;
    }
  }
  for (int j = 0; j < q; j++) {
    double w = (j & 1) ? -1.0 : 1.0;
    if (j == 0 || j == q - 1) w *= 0.5;
    out[j] = w / (t - z[j]);
    den += out[j];
  }
  for (int j = 0; j < q; j++) out[j] /= den;
}

bool q_supported(int q) { return q == 3 || q == 5 || q == 7 || q == 9 || q == 11; }

int dispatch(const fio::PlanDev &d, int kind, const void *in, void *out, int nrhs, cudaStream_t st, int stop,
             int *launches) {
  switch (d.q) {
  case 3: return fio::run_q3(d, kind, in, out, nrhs, st, stop, launches);
  case 5: return fio::run_q5(d, kind, in, out, nrhs, st, stop, launches);
  case 7: return fio::run_q7(d, kind, in, out, nrhs, st, stop, launches);
  case 9: return fio::run_q9(d, kind, in, out, nrhs, st, stop, launches);
  case 11: return fio::run_q11(d, kind, in, out, nrhs, st, stop, launches);
  }
  return (int)cudaErrorInvalidValue;
}

int check_device(fio_plan_t p) {
  int dev = -1;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return cuda_fail(e, "cudaGetDevice");
  if (dev != p->device) return fail(FIO_EINVAL, "plan was built on device %d but device %d is current", p->device, dev);
  return FIO_OK;
}

size_t elem_bytes(const fio_plan_t p) { return p->d.precision == FIO_F64 ? 16 : 8; }

}  // namespace

namespace fio {
// Lets other translation units of the library report through fio_last_error().
void set_last_error(const char *msg) { g_err = msg; }
}  // namespace fio

extern "C" {

const char *fio_last_error(void) { return g_err.c_str(); }

int fio_version(void) { return 1; }

int fio_plan(fio_plan_t *out, int N, int q, int phase_id, const double *params, int nparams, int precision,
             int nrhs_max, int s, int e) {
  using namespace fio;
  if (!out) return fail(FIO_EINVAL, "out is NULL");
  *out = nullptr;
  int L = 0;
  while ((1 << L) < N && L < 30) L++;
  if (N < 4 || N > 4096 || (1 << L) != N) return fail(FIO_EINVAL, "N=%d must be a power of two in [4, 4096]", N);
  if (!q_supported(q)) return fail(FIO_EINVAL, "q=%d not supported (compiled for 3, 5, 7, 9, 11)", q);
  if (phase_id < 0 || phase_id > 3) return fail(FIO_EINVAL, "unknown phase_id %d", phase_id);
  if (phase_id != FIO_PHASE_LINEAR && (nparams != 4 || !params))
    return fail(FIO_EINVAL, "phase %d needs 4 params, got %d", phase_id, nparams);
  if (phase_id == FIO_PHASE_LINEAR && nparams != 0 && nparams != 4)
    return fail(FIO_EINVAL, "linear phase takes no params, got %d", nparams);
  if (precision != FIO_F64 && precision != FIO_F32) return fail(FIO_EINVAL, "unknown precision %d", precision);
  if (nrhs_max < 1) return fail(FIO_EINVAL, "nrhs_max=%d must be >= 1", nrhs_max);
  if (s < 0) s = 3;
  if (s > L / 2) s = L / 2;
  if ((1 << s) > kMMax) return fail(FIO_EINVAL, "s=%d too large", s);
  if (e < 0) e = 2;
  if (e > 4) return fail(FIO_EINVAL, "e=%d must be in [0, 4]", e);
  if (phase_id == FIO_PHASE_ELLIPSE || phase_id == FIO_PHASE_CIRCLE) {
    if (params[2] == 0.0) return fail(FIO_EINVAL, "params[2] (b) must be nonzero");
  }

  int dev = 0;
  cudaError_t ce = cudaGetDevice(&dev);
  if (ce != cudaSuccess) return fail(FIO_EDEVICE, "no CUDA device: %s", cudaGetErrorString(ce));

  fio_plan_s *p = new (std::nothrow) fio_plan_s();
  static std::atomic<unsigned long long> next_serial{1};
  if (p) p->serial = next_serial++;
  if (!p) return fail(FIO_ENOMEM, "host allocation failed");
  p->device = dev;
  PlanDev &d = p->d;
  d.N = N;
  d.L = L;
  d.q = q;
  d.s = s;
  d.e = e;
  d.l0 = s;
  d.lm = L / 2;
  d.l1 = L - s;
  d.precision = precision;
  d.nrhs_max = nrhs_max;
  cudaDeviceGetAttribute(&d.smem_optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
  cudaDeviceGetAttribute(&d.num_sms, cudaDevAttrMultiProcessorCount, dev);

  d.ph = Phase();
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

  // ---- host tables
  double z[kQMax];
  cheb_grid(q, z);
  double lg[kQMax];
  memset(d.T, 0, sizeof d.T);
  for (int sg = 0; sg < 2; sg++)
    for (int jp = 0; jp < q; jp++) {
      lagrange_all(q, z, (2 * sg - 1) / 4.0 + 0.5 * z[jp], lg);
      for (int j = 0; j < q; j++) d.T[sg][j][jp] = lg[j];
    }
  memset(d.V, 0, sizeof d.V);
  const int M = 1 << s;
  for (int m = 0; m < M; m++) {
    lagrange_all(q, z, (double)m / M - 0.5, lg);
    for (int j = 0; j < q; j++) d.V[m][j] = lg[j];
  }

  std::vector<XNode> xnode;
  std::vector<P1Node> p1node;
  std::vector<P2Node> p2node;
  for (int l = 0; l <= L; l++) {
    d.tb.xoff[l] = (int)xnode.size();
    d.tb.p1off[l] = (int)p1node.size();
    d.tb.p2off[l] = (int)p2node.size();
    const double w = 1.0 / (double)(1 << l);
    for (int a = 0; a < (1 << l); a++)
      for (int j = 0; j <= q; j++) {
        XNode n;
        n.x = (a + 0.5 + (j < q ? z[j] : 0.0)) * w;
        n.s = std::sin(kTwoPi * n.x);
        n.c = std::cos(kTwoPi * n.x);
        xnode.push_back(n);
        P1Node u;
        u.p1 = n.x;
        u.rho = 0.5 * std::sqrt(2.0) * N * u.p1;
        p1node.push_back(u);
      }
    const double w2 = 1.0 / (double)(1LL << (l + e));
    for (long long b = 0; b < (1LL << (l + e)); b++)
      for (int j = 0; j <= q; j++) {
        const double p2 = (b + 0.5 + (j < q ? z[j] : 0.0)) * w2;
        P2Node v;
        v.c = std::cos(kTwoPi * p2);
        v.s = std::sin(kTwoPi * p2);
        p2node.push_back(v);
      }
  }
  std::vector<XNode> xgrid(N);
  for (int i = 0; i < N; i++) {
    xgrid[i].x = (double)i / N;
    xgrid[i].s = std::sin(kTwoPi * xgrid[i].x);
    xgrid[i].c = std::cos(kTwoPi * xgrid[i].x);
  }

  // sources sorted by their box B at level lb = L - s (eq. alg2a)
  const int lb = L - d.l0;
  const long long nb1 = 1LL << lb, nb2 = 1LL << (lb + e);
  const long long nbox = nb1 * nb2;
  const long long NN = (long long)N * N;
  std::vector<long long> boxof(NN);
  std::vector<double> P1(NN), P2(NN);
  std::vector<int> cnt(nbox + 1, 0);
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
    boxof[kf] = b1 * nb2 + b2;
    P1[kf] = p1;
    P2[kf] = ang;
    cnt[boxof[kf] + 1]++;
  }
  int maxsrc = 0;
  for (long long b = 0; b < nbox; b++) {
    maxsrc = std::max(maxsrc, cnt[b + 1]);
    cnt[b + 1] += cnt[b];
  }
  std::vector<int> pos(cnt.begin(), cnt.end() - 1);
  std::vector<Src> src(NN);
  std::vector<int> srcf(NN);
  std::vector<double> srcw(NN * 2 * q);
  for (long long kf = 0; kf < NN; kf++) {
    const int j = pos[boxof[kf]]++;
    const int k1 = (int)(kf / N) - N / 2, k2 = (int)(kf % N) - N / 2;
    Src sc;
    sc.k1 = k1;
    sc.k2 = k2;
    sc.kr = std::sqrt((double)k1 * k1 + (double)k2 * k2);
    sc.p1 = P1[kf];
    sc.c2 = std::cos(kTwoPi * P2[kf]);
    src[j] = sc;
    srcf[j] = (int)kf;
    const long long b1 = boxof[kf] / nb2, b2 = boxof[kf] % nb2;
    const double h1 = P1[kf] * (double)nb1 - (double)b1 - 0.5;
    const double h2 = P2[kf] * (double)nb2 - (double)b2 - 0.5;
    lagrange_all(q, z, h1, &srcw[(size_t)j * 2 * q]);
    lagrange_all(q, z, h2, &srcw[(size_t)j * 2 * q + q]);
  }
  d.maxsrc = maxsrc;
  d.nbox_init = (int)nbox;

  // df copies of the tables for the FP32 form (phases on the FMA pipe)
  const bool f32 = precision == FIO_F32;
  std::vector<XNodeF> xnodeF, xgridF;
  std::vector<P1NodeF> p1nodeF;
  std::vector<P2NodeF> p2nodeF;
  std::vector<SrcF> srcF;
  if (f32) {
    for (const XNode &n : xnode) xnodeF.push_back({df_split(n.x), df_split(n.s), df_split(n.c)});
    for (const XNode &n : xgrid) xgridF.push_back({df_split(n.x), df_split(n.s), df_split(n.c)});
    for (const P1Node &n : p1node) p1nodeF.push_back({df_split(n.rho)});
    for (const P2Node &n : p2node) p2nodeF.push_back({df_split(n.c), df_split(n.s)});
    for (const Src &k : src) srcF.push_back({(float)k.k1, (float)k.k2});
  }

  // ---- device: one table allocation, two state buffers
  auto al = [](size_t x) { return (x + 255) & ~(size_t)255; };
  const size_t b_x = al(xnode.size() * sizeof(XNode)), b_p1 = al(p1node.size() * sizeof(P1Node)),
               b_p2 = al(p2node.size() * sizeof(P2Node)), b_g = al(N * sizeof(XNode)), b_s = al(NN * sizeof(Src)),
               b_f = al(NN * sizeof(int)), b_w = al(srcw.size() * sizeof(double)), b_o = al((nbox + 1) * sizeof(int));
  const size_t b_xF = al(xnodeF.size() * sizeof(XNodeF)), b_gF = al(xgridF.size() * sizeof(XNodeF)),
               b_p1F = al(p1nodeF.size() * sizeof(P1NodeF)), b_p2F = al(p2nodeF.size() * sizeof(P2NodeF)),
               b_sF = al(srcF.size() * sizeof(SrcF));
  const size_t b_st = 256;  // device status word
  const size_t tbytes = b_x + b_p1 + b_p2 + b_g + b_s + b_f + b_w + b_o + b_xF + b_gF + b_p1F + b_p2F + b_sF + b_st;
  const size_t sbytes = (((size_t)NN * q * q) << e) * (size_t)nrhs_max * (precision == FIO_F64 ? 16 : 8);
  size_t freeb = 0, totalb = 0;
  cudaMemGetInfo(&freeb, &totalb);
  if (tbytes + 2 * sbytes > freeb) {
    delete p;
    return fail(FIO_ENOMEM, "plan needs %.2f GB of device memory, %.2f GB free", (tbytes + 2.0 * sbytes) / 1e9,
                freeb / 1e9);
  }
  char *tb = nullptr;
  if ((ce = cudaMalloc((void **)&tb, tbytes)) != cudaSuccess) {
    delete p;
    return cuda_fail(ce, "cudaMalloc(tables)");
  }
  p->tables = tb;
  p->table_bytes = (long long)tbytes;
  size_t off = 0;
  auto up = [&](const void *h, size_t n, size_t blk) {
    void *dptr = tb + off;
    if (n) cudaMemcpy(dptr, h, n, cudaMemcpyHostToDevice);
    off += blk;
    return dptr;
  };
  d.tb.xnode = (const XNode *)up(xnode.data(), xnode.size() * sizeof(XNode), b_x);
  d.tb.p1node = (const P1Node *)up(p1node.data(), p1node.size() * sizeof(P1Node), b_p1);
  d.tb.p2node = (const P2Node *)up(p2node.data(), p2node.size() * sizeof(P2Node), b_p2);
  d.tb.xgrid = (const XNode *)up(xgrid.data(), N * sizeof(XNode), b_g);
  d.tb.src = (const Src *)up(src.data(), NN * sizeof(Src), b_s);
  d.tb.src_f = (const int *)up(srcf.data(), NN * sizeof(int), b_f);
  d.tb.src_w = (const double *)up(srcw.data(), srcw.size() * sizeof(double), b_w);
  d.tb.box_off = (const int *)up(cnt.data(), (nbox + 1) * sizeof(int), b_o);
  {
    const int zero[64] = {0};
    d.status = (int *)up(zero, sizeof zero, b_st);
  }
  d.tf = TablesF();
  if (f32) {
    d.tf.xnode = (const XNodeF *)up(xnodeF.data(), xnodeF.size() * sizeof(XNodeF), b_xF);
    d.tf.xgrid = (const XNodeF *)up(xgridF.data(), xgridF.size() * sizeof(XNodeF), b_gF);
    d.tf.p1node = (const P1NodeF *)up(p1nodeF.data(), p1nodeF.size() * sizeof(P1NodeF), b_p1F);
    d.tf.p2node = (const P2NodeF *)up(p2nodeF.data(), p2nodeF.size() * sizeof(P2NodeF), b_p2F);
    d.tf.src = (const SrcF *)up(srcF.data(), srcF.size() * sizeof(SrcF), b_sF);
    d.tf.ph.id = phase_id;
    d.tf.ph.a = df_split(d.ph.a);
    d.tf.ph.m = df_split(d.ph.m);
    d.tf.ph.ib = df_split(d.ph.ib);
    d.tf.ph.lam = df_split(d.ph.lam);
  }
  if ((ce = cudaGetLastError()) != cudaSuccess) {
    cudaFree(tb);
    delete p;
    return cuda_fail(ce, "table upload");
  }
  for (int i = 0; i < 2; i++) {
    if ((ce = cudaMalloc(&d.state[i], sbytes)) != cudaSuccess) {
      if (i) cudaFree(d.state[0]);
      cudaFree(tb);
      delete p;
      return cuda_fail(ce, "cudaMalloc(state)");
    }
  }
  p->state_bytes = 2LL * (long long)sbytes;
  // autotune the FP32 switch on this plan's shapes (kept for every later apply)
  d.switch_impl = 0;
  d.trans_rs = 8;
  d.trans_rs_x = 8;
  d.sw_rb = 4;
  if (precision == FIO_F32) {
    int impl = 0;
    const int rc = dispatch(d, fio::RUN_TUNE, nullptr, nullptr, nrhs_max, nullptr, -1, &impl);
    if (rc) {
      fio_destroy(p);
      return cuda_fail((cudaError_t)rc, "switch autotuning");
    }
    d.switch_impl = impl;
  }
  *out = p;
  g_err.clear();
  return FIO_OK;
}

size_t fio_workspace_bytes(fio_plan_t p, int nrhs) {
  if (!p || nrhs < 1) return 0;
  const size_t eb = p->d.precision == FIO_F32 ? 8 : 16;
  return 2 * ((size_t)p->d.N * p->d.N << p->d.e) * (size_t)nrhs * p->d.q * p->d.q * eb;
}

int fio_destroy(fio_plan_t p) {
  if (!p) return FIO_OK;
  fio::batch_cache_forget(p);
  cudaDeviceSynchronize();
  if (p->d.prof) {
    for (int i = 0; i < 2 * fio::kProfSlots; i++) cudaEventDestroy(p->d.prof->ev[i]);
    delete p->d.prof;
  }
  cudaFree(p->d.state[0]);
  cudaFree(p->d.state[1]);
  cudaFree(p->tables);
  cudaFree(p->stage_buf[0]);
  cudaFree(p->stage_buf[1]);
  delete p;
  return FIO_OK;
}

static int apply_common(fio_plan_t p, int kind, const void *in, void *out, int nrhs, void *stream) {
  if (!p) return fail(FIO_EINVAL, "plan is NULL");
  if (!in || !out) return fail(FIO_EINVAL, "NULL data pointer");
  if (nrhs < 1 || nrhs > p->d.nrhs_max) return fail(FIO_EINVAL, "nrhs=%d outside [1, %d]", nrhs, p->d.nrhs_max);
  if (((uintptr_t)in | (uintptr_t)out) & 15) return fail(FIO_EINVAL, "data pointers must be 16-byte aligned");
  int rc = check_device(p);
  if (rc) return rc;
  rc = dispatch(p->d, kind, in, out, nrhs, (cudaStream_t)stream, -1, nullptr);
  if (rc) return cuda_fail((cudaError_t)rc, kind == fio::RUN_FWD ? "fio_apply" : "fio_apply_adjoint");
  return FIO_OK;
}

int fio_apply(fio_plan_t p, const void *f, void *u, int nrhs, void *stream) {
  return apply_common(p, fio::RUN_FWD, f, u, nrhs, stream);
}

int fio_apply_adjoint(fio_plan_t p, const void *g, void *fbar, int nrhs, void *stream) {
  return apply_common(p, fio::RUN_ADJ, g, fbar, nrhs, stream);
}

int fio_apply_host(fio_plan_t p, const void *in_host, void *out_host, int nrhs, int adjoint, void *stream) {
  if (!p) return fail(FIO_EINVAL, "plan is NULL");
  if (!in_host || !out_host) return fail(FIO_EINVAL, "NULL host pointer");
  if (nrhs < 1 || nrhs > p->d.nrhs_max) return fail(FIO_EINVAL, "nrhs=%d outside [1, %d]", nrhs, p->d.nrhs_max);
  int rc = check_device(p);
  if (rc) return rc;
  const size_t per = (size_t)p->d.N * p->d.N * elem_bytes(p);
  if (!p->stage_buf[0]) {
    const size_t bytes = per * p->d.nrhs_max;
    cudaError_t ce;
    for (int i = 0; i < 2; i++)
      if ((ce = cudaMalloc(&p->stage_buf[i], bytes)) != cudaSuccess) return cuda_fail(ce, "cudaMalloc(staging)");
    p->stage_bytes = bytes;
  }
  cudaStream_t st = (cudaStream_t)stream;
  const size_t n = per * nrhs;
  cudaError_t ce = cudaMemcpyAsync(p->stage_buf[0], in_host, n, cudaMemcpyHostToDevice, st);
  if (ce != cudaSuccess) return cuda_fail(ce, "cudaMemcpyAsync H2D");
  rc = apply_common(p, adjoint ? fio::RUN_ADJ : fio::RUN_FWD, p->stage_buf[0], p->stage_buf[1], nrhs, stream);
  if (rc) return rc;
  if ((ce = cudaMemcpyAsync(out_host, p->stage_buf[1], n, cudaMemcpyDeviceToHost, st)) != cudaSuccess)
    return cuda_fail(ce, "cudaMemcpyAsync D2H");
  if ((ce = cudaStreamSynchronize(st)) != cudaSuccess) return cuda_fail(ce, "cudaStreamSynchronize");
  return fio_check(p, stream);
}

int fio_debug_stage(fio_plan_t p, const void *f, int stage, void *out, void *stream) {
  if (!p || !f || !out) return fail(FIO_EINVAL, "NULL argument");
  const int nst = (p->d.lm - p->d.l0) + 2 + (p->d.l1 - p->d.lm);
  if (stage < 0 || stage >= nst) return fail(FIO_EINVAL, "stage %d outside [0, %d)", stage, nst);
  int rc = check_device(p);
  if (rc) return rc;
  rc = dispatch(p->d, fio::RUN_FWD, f, out, 1, (cudaStream_t)stream, stage, nullptr);
  if (rc) return cuda_fail((cudaError_t)rc, "fio_debug_stage");
  cudaError_t ce = cudaStreamSynchronize((cudaStream_t)stream);
  if (ce != cudaSuccess) return cuda_fail(ce, "cudaStreamSynchronize");
  return fio_check(p, stream);
}

int fio_plan_info(fio_plan_t p, fio_plan_info_t *info) {
  if (!p || !info) return fail(FIO_EINVAL, "NULL argument");
  const fio::PlanDev &d = p->d;
  info->N = d.N;
  info->L = d.L;
  info->q = d.q;
  info->s = d.s;
  info->e = d.e;
  info->l0 = d.l0;
  info->lm = d.lm;
  info->l1 = d.l1;
  info->phase_id = d.ph.id;
  info->precision = d.precision;
  info->nrhs_max = d.nrhs_max;
  info->nstages = (d.lm - d.l0) + 2 + (d.l1 - d.lm);
  info->pairs_per_level = ((long long)d.N * d.N) << d.e;
  info->state_bytes = p->state_bytes;
  info->table_bytes = p->table_bytes;
  info->max_box_sources = d.maxsrc;
  info->switch_impl = d.switch_impl;
  info->trans_rs = d.trans_rs;
  info->trans_rs_x = d.trans_rs_x;
  info->switch_rhs_tile = d.sw_rb;
  return FIO_OK;
}

int fio_profile(fio_plan_t p, int enable) {
  if (!p) return fail(FIO_EINVAL, "plan is NULL");
  int rc = check_device(p);
  if (rc) return rc;
  if (!p->d.prof) {
    fio::Prof *pr = new (std::nothrow) fio::Prof();
    if (!pr) return fail(FIO_ENOMEM, "host allocation failed");
    for (int i = 0; i < 2 * fio::kProfSlots; i++) {
      cudaError_t ce = cudaEventCreate(&pr->ev[i]);
      if (ce != cudaSuccess) {
        for (int j = 0; j < i; j++) cudaEventDestroy(pr->ev[j]);
        delete pr;
        return cuda_fail(ce, "cudaEventCreate");
      }
    }
    p->d.prof = pr;
  }
  fio::Prof *pr = p->d.prof;
  if (enable) {
    pr->n = 0;
    for (int k = 0; k < fio::kKinds; k++) {
      pr->ms[k] = 0;
      pr->launches[k] = 0;
    }
  }
  pr->enabled = enable ? 1 : 0;
  return FIO_OK;
}

int fio_profile_read(fio_plan_t p, fio_kernel_time_t *out, int max, int *n) {
  if (!p || !out || !n) return fail(FIO_EINVAL, "NULL argument");
  *n = 0;
  fio::Prof *pr = p->d.prof;
  if (!pr) return FIO_OK;
  for (int i = 0; i < pr->n; i++) {
    cudaError_t ce = cudaEventSynchronize(pr->ev[2 * i + 1]);
    if (ce != cudaSuccess) return cuda_fail(ce, "cudaEventSynchronize");
    float ms = 0.f;
    if ((ce = cudaEventElapsedTime(&ms, pr->ev[2 * i], pr->ev[2 * i + 1])) != cudaSuccess)
      return cuda_fail(ce, "cudaEventElapsedTime");
    pr->ms[pr->kind[i]] += ms;
    pr->launches[pr->kind[i]]++;
  }
  pr->n = 0;
  for (int k = 0; k < fio::kKinds && *n < max; k++) {
    if (!pr->launches[k]) continue;
    fio_kernel_time_t &o = out[(*n)++];
    snprintf(o.name, sizeof o.name, "%s", fio::kKernelNames[k]);
    o.launches = pr->launches[k];
    o.ms = pr->ms[k];
  }
  return FIO_OK;
}

int fio_check(fio_plan_t p, void *stream) {
  if (!p) return fail(FIO_EINVAL, "plan is NULL");
  int rc = check_device(p);
  if (rc) return rc;
  cudaStream_t st = (cudaStream_t)stream;
  cudaError_t ce = cudaStreamSynchronize(st);
  if (ce != cudaSuccess) return cuda_fail(ce, "cudaStreamSynchronize");
  int v = 0;
  if ((ce = cudaMemcpy(&v, p->d.status, sizeof v, cudaMemcpyDeviceToHost)) != cudaSuccess)
    return cuda_fail(ce, "cudaMemcpy(status)");
  if (v) {
    const int zero = 0;
    cudaMemcpy(p->d.status, &zero, sizeof zero, cudaMemcpyHostToDevice);
    return fail(FIO_ETIMEOUT, "a bounded device-side wait expired (status %d); results of that apply are invalid", v);
  }
  return FIO_OK;
}

int fio_plan_set_switch(fio_plan_t p, int impl) {
  if (!p) return fail(FIO_EINVAL, "plan is NULL");
  if (impl < 0 || impl > 6) return fail(FIO_EINVAL, "switch impl %d must be 0 .. 6", impl);
  if (p->d.precision != FIO_F32) return fail(FIO_EINVAL, "only FIO_F32 plans have a choice of switch kernel");
  int avail = 0;
  dispatch(p->d, fio::RUN_TC_OK, nullptr, nullptr, 1, nullptr, -1, &avail);
  if (!(avail >> impl & 1)) return fail(FIO_EINVAL, "switch kernel %d does not fit q=%d", impl, p->d.q);
  p->d.switch_impl = impl;
  return FIO_OK;
}

int fio_plan_set_wait_limit(fio_plan_t p, unsigned long long ns) {
  if (!p) return fail(FIO_EINVAL, "plan is NULL");
  p->d.handoff_ns = ns;
  return FIO_OK;
}

int fio_plan_set_tuning(fio_plan_t p, int switch_impl, int switch_rhs_tile, int trans_rs, int trans_rs_x) {
  if (!p) return fail(FIO_EINVAL, "plan is NULL");
  if (p->d.precision != FIO_F32) return fail(FIO_EINVAL, "only FIO_F32 plans are tuned");
  if (switch_rhs_tile != -1 && switch_rhs_tile != 4 && switch_rhs_tile != 8)
    return fail(FIO_EINVAL, "switch_rhs_tile %d must be 4 or 8", switch_rhs_tile);
  if (trans_rs != -1 && trans_rs != 2 && trans_rs != 4 && trans_rs != 8 && trans_rs != 32)
    return fail(FIO_EINVAL, "trans_rs %d must be 2, 4, 8 or 32", trans_rs);
  if (trans_rs_x != -1 && trans_rs_x != 2 && trans_rs_x != 4 && trans_rs_x != 8 && trans_rs_x != 32)
    return fail(FIO_EINVAL, "trans_rs_x %d must be 2, 4, 8 or 32", trans_rs_x);
  if ((trans_rs >= 32 || trans_rs_x >= 32) && p->d.q > 9)
    return fail(FIO_EINVAL, "the register-tiled translations (trans_rs 32) are compiled for q <= 9");
  if (switch_impl != -1) {
    const int rc = fio_plan_set_switch(p, switch_impl);
    if (rc) return rc;
  }
  if (switch_rhs_tile != -1) p->d.sw_rb = switch_rhs_tile;
  if (trans_rs != -1) p->d.trans_rs = trans_rs;
  if (trans_rs_x != -1) p->d.trans_rs_x = trans_rs_x;
  return FIO_OK;
}

int fio_kernel_launches(fio_plan_t p, int nrhs, int adjoint) {
  if (!p) return fail(FIO_EINVAL, "plan is NULL");
  int n = 0;
  dispatch(p->d, adjoint ? fio::RUN_COUNT_ADJ : fio::RUN_COUNT_FWD, nullptr, nullptr, nrhs, nullptr, -1, &n);
  return n;
}

}  // extern "C"
