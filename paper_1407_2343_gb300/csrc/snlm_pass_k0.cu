// Pass and patch-distance kernels for patch half-width K = 0.
#include "snlm_pass_tma.cuh"

SNLM_INSTANTIATE_K(0)
SNLM_INSTANTIATE_TMA_K(0)
