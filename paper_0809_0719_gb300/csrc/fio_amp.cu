// fio_amp.cu -- variable amplitudes (eq. allfio): u(x) = sum_k a(x,k) e^{2 pi i Phi(x,k)} f(k)
// with a separated amplitude a(x,k) = sum_t g_t(x) h_t(k).  As the paper suggests, the
// terms f_t = h_t f are the right-hand sides of ONE vectorised butterfly, so every phase
// evaluation is shared by all of them; then u = sum_t g_t (B f_t).  The adjoint applies
// the conjugate transpose of the same three steps in reverse order.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdarg>
#include <cstdio>

#include "fio.h"
#include "fio_internal.cuh"

namespace {

using namespace fio;

int mfail(int code, const char *fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof buf, fmt, ap);
  va_end(ap);
  set_last_error(buf);
  return code;
}

template <typename CT> __device__ __forceinline__ CT cmulz(CT a, CT b, bool conj_a) {
  CT r;
  const auto ay = conj_a ? -a.y : a.y;
  r.x = a.x * b.x - ay * b.y;
  r.y = a.x * b.y + ay * b.x;
  return r;
}

// rhs[r * nt + t][i] = w_t[i] (or conj w_t[i]) * x[r][i]
template <typename CT>
__global__ void k_amp_spread(const CT *__restrict__ x, const CT *__restrict__ w, int nt, int nrhs, long long NN,
                             bool conj_w, CT *__restrict__ rhs) {
  const long long n = (long long)nrhs * nt * NN;
  for (long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x; idx < n; idx += (long long)gridDim.x * blockDim.x) {
    const long long i = idx % NN, rt = idx / NN;
    const int t = (int)(rt % nt), r = (int)(rt / nt);
    rhs[idx] = cmulz(w[(long long)t * NN + i], x[(long long)r * NN + i], conj_w);
  }
}

// y[r][i] = sum_t w_t[i] (or conj w_t[i]) * v[r * nt + t][i], t in increasing order
template <typename CT>
__global__ void k_amp_gather(const CT *__restrict__ v, const CT *__restrict__ w, int nt, int nrhs, long long NN,
                             bool conj_w, CT *__restrict__ y) {
  const long long n = (long long)nrhs * NN;
  for (long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x; idx < n; idx += (long long)gridDim.x * blockDim.x) {
    const long long i = idx % NN;
    const int r = (int)(idx / NN);
    CT acc;
    acc.x = 0;
    acc.y = 0;
    for (int t = 0; t < nt; t++) {
      const CT p = cmulz(w[(long long)t * NN + i], v[((long long)r * nt + t) * NN + i], conj_w);
      acc.x += p.x;
      acc.y += p.y;
    }
    y[idx] = acc;
  }
}

template <typename CT>
int amp_run(fio_plan_t p, const void *in, const void *g, const void *h, int nt, void *out, int nrhs, int adjoint,
            cudaStream_t st) {
  const long long NN = (long long)p->d.N * p->d.N;
  const int grid = 4 * std::max(1, p->d.num_sms), block = 256;
  CT *rhs = (CT *)p->stage_buf[0], *res = (CT *)p->stage_buf[1];
  // forward: f_t = h_t f, then u = sum_t g_t B f_t;  adjoint: v_t = conj(g_t) gin, then fbar = sum_t conj(h_t) B^H v_t
  k_amp_spread<CT><<<grid, block, 0, st>>>((const CT *)in, (const CT *)(adjoint ? g : h), nt, nrhs, NN, adjoint != 0, rhs);
  cudaError_t ce = cudaGetLastError();
  if (ce != cudaSuccess) return mfail(FIO_ECUDA, "amplitude spread: %s", cudaGetErrorString(ce));
  int rc = adjoint ? fio_apply_adjoint(p, rhs, res, nrhs * nt, st) : fio_apply(p, rhs, res, nrhs * nt, st);
  if (rc) return rc;
  k_amp_gather<CT><<<grid, block, 0, st>>>(res, (const CT *)(adjoint ? h : g), nt, nrhs, NN, adjoint != 0, (CT *)out);
  ce = cudaGetLastError();
  return ce == cudaSuccess ? FIO_OK : mfail(FIO_ECUDA, "amplitude gather: %s", cudaGetErrorString(ce));
}

}  // namespace

extern "C" {

int fio_apply_amplitude(fio_plan_t p, const void *in, const void *g, const void *h, int nt, void *out, int nrhs,
                        int adjoint, void *stream) {
  if (!p) return mfail(FIO_EINVAL, "plan is NULL");
  if (!in || !g || !h || !out) return mfail(FIO_EINVAL, "NULL data pointer");
  if (nt < 1 || nrhs < 1 || (long long)nt * nrhs > p->d.nrhs_max)
    return mfail(FIO_EINVAL, "nt=%d times nrhs=%d must be in [1, nrhs_max=%d]", nt, nrhs, p->d.nrhs_max);
  int dev = -1;
  cudaGetDevice(&dev);
  if (dev != p->device) return mfail(FIO_EINVAL, "plan was built on device %d but device %d is current", p->device, dev);
  const size_t eb = p->d.precision == FIO_F64 ? 16 : 8;
  if (!p->stage_buf[0]) {  // the plan's staging buffers hold the nt nrhs right-hand sides and results
    const size_t bytes = (size_t)p->d.N * p->d.N * eb * p->d.nrhs_max;
    for (int i = 0; i < 2; i++) {
      const cudaError_t ce = cudaMalloc(&p->stage_buf[i], bytes);
      if (ce != cudaSuccess) return mfail(FIO_ENOMEM, "cudaMalloc(staging): %s", cudaGetErrorString(ce));
    }
    p->stage_bytes = bytes;
  }
  cudaStream_t st = (cudaStream_t)stream;
  return p->d.precision == FIO_F64 ? amp_run<double2>(p, in, g, h, nt, out, nrhs, adjoint, st)
                                   : amp_run<float2>(p, in, g, h, nt, out, nrhs, adjoint, st);
}

}  // extern "C"
