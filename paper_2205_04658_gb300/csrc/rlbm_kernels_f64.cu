// Kernels of the double storage type.
#include "rlbm_kernels.cuh"
RLBM_DEFINE_LAUNCHERS(double, f64)
