// Pass and patch-distance kernels for patch half-width K = 5.
#include "snlm_pass_tma.cuh"

SNLM_INSTANTIATE_K(5)
SNLM_INSTANTIATE_TMA_K(5)
