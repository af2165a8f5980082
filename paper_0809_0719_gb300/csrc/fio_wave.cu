// fio_wave.cu -- the wave-equation solution operator as a sum of two FIOs (Sec. 1):
//     u = w_plus B_plus f + w_minus B_minus f,
// e.g. the phases x.k + c|k|t and x.k - c|k|t with weights 1/2 for u_tt = c^2 Lap u with
// u_t(x, 0) = 0 and f the Fourier coefficients of u(x, 0).  Each FIO runs through its own
// plan; the second result goes to the minus plan's staging buffer and one kernel forms the
// weighted sum.  The adjoint is the same sum of the two adjoints (real weights).
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdarg>
#include <cstdio>

#include "fio.h"
#include "fio_internal.cuh"

namespace {

using namespace fio;

int wfail(int code, const char *fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof buf, fmt, ap);
  va_end(ap);
  set_last_error(buf);
  return code;
}

// y[i] = wp y[i] + wm v[i] over n complex elements
template <typename CT, typename R>
__global__ void k_wave_sum(CT *__restrict__ y, const CT *__restrict__ v, R wp, R wm, long long n) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    const CT a = y[i], b = v[i];
    CT r;
    r.x = wp * a.x + wm * b.x;
    r.y = wp * a.y + wm * b.y;
    y[i] = r;
  }
}

int run_any(const PlanDev &d, int kind, const void *in, void *out, int nrhs, cudaStream_t st) {
  switch (d.q) {
  case 3: return run_q3(d, kind, in, out, nrhs, st, -1, nullptr);
  case 5: return run_q5(d, kind, in, out, nrhs, st, -1, nullptr);
  case 7: return run_q7(d, kind, in, out, nrhs, st, -1, nullptr);
  case 9: return run_q9(d, kind, in, out, nrhs, st, -1, nullptr);
  case 11: return run_q11(d, kind, in, out, nrhs, st, -1, nullptr);
  }
  return (int)cudaErrorInvalidValue;
}

// The c(x)|k| phase lambda x.k + s t (a + m sin 2 pi x1 sin 2 pi x2)|k| / b (s = +-1) on a
// copy of the plan's device description: the node, source and Lagrange tables do not
// depend on the phase, only the kernels' Phase arguments do.
void set_wave_phase(PlanDev &d, const Phase &base, double sign_t) {
  d.ph = base;
  d.ph.a = base.a * sign_t;
  d.ph.m = base.m * sign_t;
  if (d.precision == FIO_F32) {
    d.tf.ph.id = d.ph.id;
    d.tf.ph.a = df_split(d.ph.a);
    d.tf.ph.m = df_split(d.ph.m);
    d.tf.ph.ib = df_split(d.ph.ib);
    d.tf.ph.lam = df_split(d.ph.lam);
  }
}

}  // namespace

extern "C" {

int fio_apply_wave(fio_plan_t plus, fio_plan_t minus, const void *in, void *out, int nrhs, double w_plus,
                   double w_minus, int adjoint, void *stream) {
  if (!plus || !minus) return wfail(FIO_EINVAL, "plan is NULL");
  if (!in || !out) return wfail(FIO_EINVAL, "NULL data pointer");
  if (in == out) return wfail(FIO_EINVAL, "in and out must be different buffers");
  if (plus->d.N != minus->d.N || plus->d.precision != minus->d.precision)
    return wfail(FIO_EINVAL, "the two plans differ in N (%d, %d) or precision", plus->d.N, minus->d.N);
  if (plus->device != minus->device) return wfail(FIO_EINVAL, "the two plans live on different devices");
  if (nrhs < 1 || nrhs > std::min(plus->d.nrhs_max, minus->d.nrhs_max))
    return wfail(FIO_EINVAL, "nrhs=%d must be in [1, %d]", nrhs, std::min(plus->d.nrhs_max, minus->d.nrhs_max));
  int dev = -1;
  cudaGetDevice(&dev);
  if (dev != plus->device) return wfail(FIO_EINVAL, "plans were built on device %d but device %d is current", plus->device, dev);
  const bool f64 = plus->d.precision == FIO_F64;
  const size_t eb = f64 ? 16 : 8;
  const long long n = (long long)nrhs * plus->d.N * plus->d.N;
  if (!minus->stage_buf[0]) {  // the minus plan's staging buffers (nrhs_max N^2 elements each)
    const size_t bytes = (size_t)minus->d.N * minus->d.N * eb * minus->d.nrhs_max;
    for (int i = 0; i < 2; i++) {
      const cudaError_t ce = cudaMalloc(&minus->stage_buf[i], bytes);
      if (ce != cudaSuccess) return wfail(FIO_ENOMEM, "cudaMalloc(staging): %s", cudaGetErrorString(ce));
    }
    minus->stage_bytes = bytes;
  }
  void *tmp = minus->stage_buf[0];
  int rc = adjoint ? fio_apply_adjoint(plus, in, out, nrhs, stream) : fio_apply(plus, in, out, nrhs, stream);
  if (rc) return rc;
  rc = adjoint ? fio_apply_adjoint(minus, in, tmp, nrhs, stream) : fio_apply(minus, in, tmp, nrhs, stream);
  if (rc) return rc;
  const cudaStream_t st = (cudaStream_t)stream;
  const int grid = 4 * std::max(1, plus->d.num_sms), block = 256;
  if (f64)
    k_wave_sum<double2, double><<<grid, block, 0, st>>>((double2 *)out, (const double2 *)tmp, w_plus, w_minus, n);
  else
    k_wave_sum<float2, float><<<grid, block, 0, st>>>((float2 *)out, (const float2 *)tmp, (float)w_plus, (float)w_minus, n);
  const cudaError_t ce = cudaGetLastError();
  return ce == cudaSuccess ? FIO_OK : wfail(FIO_ECUDA, "wave sum: %s", cudaGetErrorString(ce));
}

}  // extern "C"

extern "C" int fio_apply_wave_series(fio_plan_t plan, const double *times, int ntimes, const void *in, void *out,
                                     int nrhs, void *stream) {
  if (!plan) return wfail(FIO_EINVAL, "plan is NULL");
  if (plan->d.ph.id != FIO_PHASE_CIRCLE) return wfail(FIO_EINVAL, "fio_apply_wave_series needs a FIO_PHASE_CIRCLE plan");
  if (!times || ntimes < 1) return wfail(FIO_EINVAL, "need ntimes >= 1 times");
  if (!in || !out) return wfail(FIO_EINVAL, "NULL data pointer");
  if (((uintptr_t)in | (uintptr_t)out) & 15) return wfail(FIO_EINVAL, "data pointers must be 16-byte aligned");
  if (nrhs < 1 || nrhs > plan->d.nrhs_max) return wfail(FIO_EINVAL, "nrhs=%d must be in [1, %d]", nrhs, plan->d.nrhs_max);
  int dev = -1;
  cudaGetDevice(&dev);
  if (dev != plan->device) return wfail(FIO_EINVAL, "plan was built on device %d but device %d is current", plan->device, dev);
  const bool f64 = plan->d.precision == FIO_F64;
  const size_t eb = f64 ? 16 : 8;
  const long long n = (long long)nrhs * plan->d.N * plan->d.N;
  if ((const char *)in < (const char *)out + (size_t)ntimes * n * eb && (const char *)out < (const char *)in + n * eb)
    return wfail(FIO_EINVAL, "in and out overlap");
  if (!plan->stage_buf[0]) {  // the plan's staging buffers (nrhs_max N^2 elements each)
    const size_t bytes = (size_t)plan->d.N * plan->d.N * eb * plan->d.nrhs_max;
    for (int i = 0; i < 2; i++) {
      const cudaError_t ce = cudaMalloc(&plan->stage_buf[i], bytes);
      if (ce != cudaSuccess) return wfail(FIO_ENOMEM, "cudaMalloc(staging): %s", cudaGetErrorString(ce));
    }
    plan->stage_bytes = bytes;
  }
  const cudaStream_t st = (cudaStream_t)stream;
  const int grid = 4 * std::max(1, plan->d.num_sms), block = 256;
  PlanDev d = plan->d;  // phases change per launch; tables and state buffers are the plan's
  void *tmp = plan->stage_buf[0];
  for (int k = 0; k < ntimes; k++) {
    char *uk = (char *)out + (size_t)k * n * eb;
    set_wave_phase(d, plan->d.ph, times[k]);
    int rc = run_any(d, RUN_FWD, in, uk, nrhs, st);
    if (rc) return wfail(FIO_ECUDA, "wave series, B+ at t=%g: %s", times[k], cudaGetErrorString((cudaError_t)rc));
    set_wave_phase(d, plan->d.ph, -times[k]);
    rc = run_any(d, RUN_FWD, in, tmp, nrhs, st);
    if (rc) return wfail(FIO_ECUDA, "wave series, B- at t=%g: %s", times[k], cudaGetErrorString((cudaError_t)rc));
    if (f64)
      k_wave_sum<double2, double><<<grid, block, 0, st>>>((double2 *)uk, (const double2 *)tmp, 0.5, 0.5, n);
    else
      k_wave_sum<float2, float><<<grid, block, 0, st>>>((float2 *)uk, (const float2 *)tmp, 0.5f, 0.5f, n);
    const cudaError_t ce = cudaGetLastError();
    if (ce != cudaSuccess) return wfail(FIO_ECUDA, "wave sum: %s", cudaGetErrorString(ce));
  }
  return FIO_OK;
}
