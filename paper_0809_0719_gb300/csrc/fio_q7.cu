// fio_q7.cu -- the butterfly kernels instantiated for q = 7 (both precisions).
#include "fio_run.cuh"

namespace fio {
int run_q7(const PlanDev &p, int kind, const void *in, void *out, int nrhs, cudaStream_t st, int stop, int *launches) {
  return p.precision == 0 ? run_plan<double, 7>(p, kind, in, out, nrhs, st, stop, launches)
                          : run_plan<float, 7>(p, kind, in, out, nrhs, st, stop, launches);
}
}  // namespace fio
