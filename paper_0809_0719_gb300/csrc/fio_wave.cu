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
