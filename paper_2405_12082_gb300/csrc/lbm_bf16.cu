// lbm_bf16.cu -- kernels for LBM_BF16 population storage.
#include "lbm_kernels.cuh"

LBM_INSTANTIATE(LBM_BF16)
