// fio_q9.cu -- the butterfly kernels instantiated for q = 9 (both precisions).
#include "fio_run.cuh"

namespace fio {
int run_q9(const PlanDev &p, int kind, const void *in, void *out, int nrhs, cudaStream_t st, int stop, int *launches) {
  return p.precision == 0 ? run_plan<double, 9>(p, kind, in, out, nrhs, st, stop, launches)
                          : run_plan<float, 9>(p, kind, in, out, nrhs, st, stop, launches);
}
}  // namespace fio
