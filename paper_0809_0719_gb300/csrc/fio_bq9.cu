// fio_bq9.cu -- the batched (many-plan) kernels instantiated for q = 9.
#include "fio_batch.cuh"

namespace fio {
int batch_q9(const BLaunch &L, cudaStream_t st, int smem_optin, int *blocks_per_sm, int *block) {
  return batch_launch<9>(L, st, smem_optin, blocks_per_sm, block);
}
}  // namespace fio
