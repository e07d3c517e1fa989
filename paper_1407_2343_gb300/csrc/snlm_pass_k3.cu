// Pass and patch-distance kernels for patch half-width K = 3.
#include "snlm_pass_tma.cuh"

SNLM_INSTANTIATE_K(3)
SNLM_INSTANTIATE_TMA_K(3)
