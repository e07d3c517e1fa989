// Pass and patch-distance kernels for patch half-width K = 7.
#include "snlm_pass_tma.cuh"

SNLM_INSTANTIATE_K(7)
SNLM_INSTANTIATE_TMA_K(7)
