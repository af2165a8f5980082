// fio_q11.cu -- the butterfly kernels instantiated for q = 11 (both precisions).
#include "fio_run.cuh"

namespace fio {
int run_q11(const PlanDev &p, int kind, const void *in, void *out, int nrhs, cudaStream_t st, int stop, int *launches) {
  return p.precision == 0 ? run_plan<double, 11>(p, kind, in, out, nrhs, st, stop, launches)
                          : run_plan<float, 11>(p, kind, in, out, nrhs, st, stop, launches);
}
}  // namespace fio
