// Kernels of the float storage type.
#include "rlbm_kernels.cuh"
RLBM_DEFINE_LAUNCHERS(float, f32)
