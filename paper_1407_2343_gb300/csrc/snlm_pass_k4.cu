// Pass and patch-distance kernels for patch half-width K = 4.
#include "snlm_pass_tma.cuh"

SNLM_INSTANTIATE_K(4)
SNLM_INSTANTIATE_TMA_K(4)
