// ibm_batch_f16.cu -- the batched serving kernel for one storage precision
// (PREC_FP16_DEV); see ibm_batch.cuh.
#include "ibm_batch.cuh"

template struct ibm::BatchOps<ibm::PREC_FP16_DEV>;
