// fio_q5.cu -- the butterfly kernels instantiated for q = 5 (both precisions).
#include "fio_run.cuh"

namespace fio {
int run_q5(const PlanDev &p, int kind, const void *in, void *out, int nrhs, cudaStream_t st, int stop, int *launches) {
  return p.precision == 0 ? run_plan<double, 5>(p, kind, in, out, nrhs, st, stop, launches)
                          : run_plan<float, 5>(p, kind, in, out, nrhs, st, stop, launches);
}
}  // namespace fio
