// Pass and patch-distance kernels for patch half-width K = 6.
#include "snlm_pass_impl.cuh"

SNLM_INSTANTIATE_K(6)
