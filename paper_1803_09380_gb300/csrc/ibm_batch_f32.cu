// ibm_batch_f32.cu -- the batched serving kernel for one storage precision
// (PREC_FP32); see ibm_batch.cuh.
#include "ibm_batch.cuh"

template struct ibm::BatchOps<ibm::PREC_FP32>;
