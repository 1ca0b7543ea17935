// Kernels of the __nv_bfloat16 storage type.
#include "rlbm_kernels.cuh"
RLBM_DEFINE_LAUNCHERS(__nv_bfloat16, bf16)
