// Batched persistent class kernel for patch half-width K = 1.
#include "snlm_batch_impl.cuh"

SNLM_INSTANTIATE_BATCH_K(1)
