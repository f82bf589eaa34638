// lbm_staged_bf16.cu -- staged step kernels for LBM_BF16 population storage.
#include "lbm_staged.cuh"

LBM_INSTANTIATE_STAGED(LBM_BF16)
