// fio_internal.cuh -- the plan object behind fio_plan_t and the per-q entry
// points shared by the library's translation units (not part of the C ABI).
#pragma once
#include "fio_run.cuh"

struct fio_plan_s {
  fio::PlanDev d;
  int device;
  void *tables;
  long long table_bytes, state_bytes;
  void *stage_buf[2];
  size_t stage_bytes;
};

namespace fio {
int run_q3(const PlanDev &, int, const void *, void *, int, cudaStream_t, int, int *);
int run_q5(const PlanDev &, int, const void *, void *, int, cudaStream_t, int, int *);
int run_q7(const PlanDev &, int, const void *, void *, int, cudaStream_t, int, int *);
int run_q9(const PlanDev &, int, const void *, void *, int, cudaStream_t, int, int *);
int run_q11(const PlanDev &, int, const void *, void *, int, cudaStream_t, int, int *);
void set_last_error(const char *msg);
}  // namespace fio
