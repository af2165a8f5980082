// fio_auto.cu -- the sampled direct sum on the GPU (fio_direct) and the choice of q
// from a target accuracy (fio_plan_auto): the error of the butterfly falls
// geometrically with q (Sec. 5), so q is raised until the relative L2 error of
// eq. err, estimated on seeded sample points against the direct sum, meets the target.
#include <cuda_runtime.h>

#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <vector>

#include "fio.h"
#include "fio_internal.cuh"

namespace {

using namespace fio;

int afail(int code, const char *fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof buf, fmt, ap);
  va_end(ap);
  set_last_error(buf);
  return code;
}

constexpr int kDirectThreads = 256;

// u(x) = sum_k e^{2 pi i Phi(x,k)} f(k) at the flat grid indices xi (eq. dfio), one CTA per
// (sample, RHS).  Terms in the order of the plan's sorted source list, each thread a
// fixed strided subset, accumulated in FP64, then a fixed-order tree: the result is
// independent of timing.  FP32 plans evaluate Phi in double-float (as their butterfly
// does), FP64 plans in FP64.
template <typename CT>
__global__ void __launch_bounds__(kDirectThreads) k_direct(Tables tb, TablesF tf, Phase ph, int L, const CT *__restrict__ f,
                                                          const long long *__restrict__ xi, int nx,
                                                          double2 *__restrict__ out) {
  __shared__ double2 red[kDirectThreads];
  const long long NN = 1LL << (2 * L);
  const int s = blockIdx.x, r = blockIdx.y;
  const long long x = xi[s];
  const int i1 = (int)(x >> L), i2 = (int)(x & ((1LL << L) - 1));
  const CT *fr = f + (long long)r * NN;
  const bool fast = sizeof(CT) == 8 && tf.xnode != nullptr && ph.id != 3;
  XDesc xd;
  if (fast) xd = xdesc(tf.ph, tf.xgrid[i1], tf.xgrid[i2]);
  double ax = 0.0, ay = 0.0;
  for (long long j = threadIdx.x; j < NN; j += blockDim.x) {
    double ex, ey;
    if (fast) {
      const float2 e = expi_df(theta_k(tf.ph, xd, tf.src[j].k1, tf.src[j].k2));
      ex = e.x;
      ey = e.y;
    } else {
      const double2 e = expi<double>(theta_xk(ph, tb.xgrid[i1], tb.xgrid[i2], tb.src[j]));
      ex = e.x;
      ey = e.y;
    }
    const CT v = fr[tb.src_f[j]];
    const double vx = v.x, vy = v.y;
    ax = fma(ex, vx, fma(-ey, vy, ax));
    ay = fma(ex, vy, fma(ey, vx, ay));
  }
  red[threadIdx.x] = make_double2(ax, ay);
  __syncthreads();
  for (int w = kDirectThreads / 2; w > 0; w >>= 1) {
    if (threadIdx.x < w) {
      red[threadIdx.x].x += red[threadIdx.x + w].x;
      red[threadIdx.x].y += red[threadIdx.x + w].y;
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) out[(long long)r * nx + s] = red[0];
}

// Seeded host generator for the probe input of fio_plan_auto: splitmix64 words mapped to
// uniforms in (0,1), pairs turned into standard normals by the Box-Muller transform.
struct Rng {
  unsigned long long s;
  unsigned long long next() {
    unsigned long long z = (s += 0x9E3779B97F4A7C15ULL);
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
    return z ^ (z >> 31);
  }
  double uniform() { return ((next() >> 11) + 0.5) * (1.0 / 9007199254740992.0); }
  void normal2(double &a, double &b) {
    const double r = std::sqrt(-2.0 * std::log(uniform())), t = 6.283185307179586 * uniform();
    a = r * std::cos(t);
    b = r * std::sin(t);
  }
};

}  // namespace

extern "C" {

int fio_direct(fio_plan_t p, const void *f, int nrhs, const long long *xi, int nx, void *out, void *stream) {
  if (!p || !f || !xi || !out) return afail(FIO_EINVAL, "NULL argument");
  if (nrhs < 1 || nx < 1) return afail(FIO_EINVAL, "nrhs=%d and nx=%d must be >= 1", nrhs, nx);
  if (nrhs > 65535) return afail(FIO_EINVAL, "nrhs=%d above 65535", nrhs);
  int dev = -1;
  cudaGetDevice(&dev);
  if (dev != p->device) return afail(FIO_EINVAL, "plan was built on device %d but device %d is current", p->device, dev);
  const PlanDev &d = p->d;
  cudaStream_t st = (cudaStream_t)stream;
  dim3 grid((unsigned)nx, (unsigned)nrhs);
  if (d.precision == FIO_F64)
    k_direct<double2><<<grid, kDirectThreads, 0, st>>>(d.tb, d.tf, d.ph, d.L, (const double2 *)f, xi, nx, (double2 *)out);
  else
    k_direct<float2><<<grid, kDirectThreads, 0, st>>>(d.tb, d.tf, d.ph, d.L, (const float2 *)f, xi, nx, (double2 *)out);
  const cudaError_t ce = cudaGetLastError();
  if (ce != cudaSuccess) return afail(FIO_ECUDA, "fio_direct: %s", cudaGetErrorString(ce));
  return FIO_OK;
}

int fio_plan_auto(fio_plan_t *out, int N, int phase_id, const double *params, int nparams, int precision, int nrhs_max,
                  int s, int e, double target, int nsample, unsigned long long seed, int *q_out, double *err_out) {
  if (!out) return afail(FIO_EINVAL, "out is NULL");
  *out = nullptr;
  if (N < 4 || N > 4096 || (N & (N - 1))) return afail(FIO_EINVAL, "N=%d must be a power of two in [4, 4096]", N);
  if (!(target > 0.0)) return afail(FIO_EINVAL, "target %g must be positive", target);
  if (nsample < 1 || (long long)nsample > (long long)N * N)
    return afail(FIO_EINVAL, "nsample=%d outside [1, N^2]", nsample);
  static const int qs[] = {3, 5, 7, 9, 11};
  const long long NN = (long long)N * N;
  const size_t eb = precision == FIO_F64 ? 16 : 8;
  // probe input (complex white noise) and distinct sample points, both from the seed
  Rng rng{seed};
  std::vector<double> fh(2 * NN);
  for (long long k = 0; k < NN; k++) rng.normal2(fh[2 * k], fh[2 * k + 1]);
  std::vector<float> ff;
  if (precision != FIO_F64) {
    ff.resize(2 * NN);
    for (long long k = 0; k < 2 * NN; k++) ff[k] = (float)fh[k];
  }
  std::vector<long long> xi;
  {
    std::vector<char> used(NN, 0);
    while ((int)xi.size() < nsample) {
      const long long x = (long long)(rng.next() % (unsigned long long)NN);
      if (!used[x]) {
        used[x] = 1;
        xi.push_back(x);
      }
    }
  }
  void *df_ = nullptr, *du = nullptr, *dref = nullptr;
  long long *dxi = nullptr;
  cudaError_t ce = cudaMalloc(&df_, NN * eb);
  if (ce == cudaSuccess) ce = cudaMalloc(&du, NN * eb);
  if (ce == cudaSuccess) ce = cudaMalloc(&dref, nsample * sizeof(double2));
  if (ce == cudaSuccess) ce = cudaMalloc((void **)&dxi, nsample * sizeof(long long));
  if (ce == cudaSuccess)
    ce = cudaMemcpy(df_, precision == FIO_F64 ? (const void *)fh.data() : (const void *)ff.data(), NN * eb,
                    cudaMemcpyHostToDevice);
  if (ce == cudaSuccess) ce = cudaMemcpy(dxi, xi.data(), nsample * sizeof(long long), cudaMemcpyHostToDevice);
  int rc = ce == cudaSuccess ? FIO_OK : afail(ce == cudaErrorMemoryAllocation ? FIO_ENOMEM : FIO_ECUDA, "%s",
                                            cudaGetErrorString(ce));
  std::vector<double> ref(2 * nsample);
  std::vector<unsigned char> uh(NN * eb);
  fio_plan_t best = nullptr;
  int best_q = 0;
  double best_err = INFINITY;
  bool have_ref = false;
  for (int qi = 0; qi < 5 && rc == FIO_OK; qi++) {
    fio_plan_t p = nullptr;
    rc = fio_plan(&p, N, qs[qi], phase_id, params, nparams, precision, nrhs_max, s, e);
    if (rc) break;
    if (!have_ref) {  // the direct sum does not depend on q
      if ((rc = fio_direct(p, df_, 1, dxi, nsample, dref, nullptr)) != FIO_OK) {
        fio_destroy(p);
        break;
      }
      if ((ce = cudaMemcpy(ref.data(), dref, nsample * sizeof(double2), cudaMemcpyDeviceToHost)) != cudaSuccess) {
        rc = afail(FIO_ECUDA, "%s", cudaGetErrorString(ce));
        fio_destroy(p);
        break;
      }
      have_ref = true;
    }
    if ((rc = fio_apply(p, df_, du, 1, nullptr)) != FIO_OK ||
        (ce = cudaMemcpy(uh.data(), du, NN * eb, cudaMemcpyDeviceToHost)) != cudaSuccess) {
      if (!rc) rc = afail(FIO_ECUDA, "%s", cudaGetErrorString(ce));
      fio_destroy(p);
      break;
    }
    double num = 0.0, den = 0.0;  // eq. err on the sample
    for (int k = 0; k < nsample; k++) {
      double ux, uy;
      if (precision == FIO_F64) {
        ux = ((const double *)uh.data())[2 * xi[k]];
        uy = ((const double *)uh.data())[2 * xi[k] + 1];
      } else {
        ux = ((const float *)uh.data())[2 * xi[k]];
        uy = ((const float *)uh.data())[2 * xi[k] + 1];
      }
      const double dx = ux - ref[2 * k], dy = uy - ref[2 * k + 1];
      num += dx * dx + dy * dy;
      den += ref[2 * k] * ref[2 * k] + ref[2 * k + 1] * ref[2 * k + 1];
    }
    const double err = den > 0.0 ? std::sqrt(num / den) : 0.0;
    if (best) fio_destroy(best);
    best = p;
    best_q = qs[qi];
    best_err = err;
    if (err <= target) break;
  }
  cudaFree(df_);
  cudaFree(du);
  cudaFree(dref);
  cudaFree(dxi);
  if (rc != FIO_OK) {
    if (best) fio_destroy(best);
    return rc;
  }
  *out = best;
  if (q_out) *q_out = best_q;
  if (err_out) *err_out = best_err;
  set_last_error(best_err <= target ? "" : "target accuracy not reached with q = 11; the q = 11 plan is returned");
  return FIO_OK;
}

}  // extern "C"
