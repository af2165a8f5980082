// fio_bq11.cu -- the batched (many-plan) kernels instantiated for q = 11.
#include "fio_batch.cuh"

namespace fio {
int batch_q11(const BLaunch &L, cudaStream_t st, int smem_optin, int *blocks_per_sm, int *block) {
  return batch_launch<11>(L, st, smem_optin, blocks_per_sm, block);
}
}  // namespace fio
