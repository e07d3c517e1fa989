// Batched persistent class kernel for patch half-width K = 5.
#include "snlm_batch_impl.cuh"

SNLM_INSTANTIATE_BATCH_K(5)
