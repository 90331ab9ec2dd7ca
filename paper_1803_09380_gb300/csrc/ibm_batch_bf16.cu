// ibm_batch_bf16.cu -- the batched serving kernel for one storage precision
// (PREC_BF16_DEV); see ibm_batch.cuh.
#include "ibm_batch.cuh"

template struct ibm::BatchOps<ibm::PREC_BF16_DEV>;
