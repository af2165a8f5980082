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
  unsigned long long serial;  // unique per plan in this process (keys fio_apply_batch's cache)
};

namespace fio {
int run_q3(const PlanDev &, int, const void *, void *, int, cudaStream_t, int, int *);
int run_q5(const PlanDev &, int, const void *, void *, int, cudaStream_t, int, int *);
int run_q7(const PlanDev &, int, const void *, void *, int, cudaStream_t, int, int *);
int run_q9(const PlanDev &, int, const void *, void *, int, cudaStream_t, int, int *);
int run_q11(const PlanDev &, int, const void *, void *, int, cudaStream_t, int, int *);
void set_last_error(const char *msg);
void batch_cache_forget(fio_plan_t p);  // drop fio_apply_batch's batches that use p
}  // namespace fio
