// Pass and patch-distance kernels for patch half-width K = 2.
#include "snlm_pass_tma.cuh"

SNLM_INSTANTIATE_K(2)
SNLM_INSTANTIATE_TMA_K(2)
