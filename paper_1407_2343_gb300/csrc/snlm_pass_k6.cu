// Pass and patch-distance kernels for patch half-width K = 6.
#include "snlm_pass_tma.cuh"

SNLM_INSTANTIATE_K(6)
SNLM_INSTANTIATE_TMA_K(6)
