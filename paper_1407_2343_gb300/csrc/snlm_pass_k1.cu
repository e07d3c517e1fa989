// Pass and patch-distance kernels for patch half-width K = 1.
#include "snlm_pass_tma.cuh"

SNLM_INSTANTIATE_K(1)
SNLM_INSTANTIATE_TMA_K(1)
