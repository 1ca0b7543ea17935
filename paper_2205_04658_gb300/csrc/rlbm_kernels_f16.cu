// Kernels of the __half storage type.
#include "rlbm_kernels.cuh"
RLBM_DEFINE_LAUNCHERS(__half, f16)
