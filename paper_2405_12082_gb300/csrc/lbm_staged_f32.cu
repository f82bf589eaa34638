// lbm_staged_f32.cu -- staged step kernels for LBM_F32 population storage.
#include "lbm_staged.cuh"

LBM_INSTANTIATE_STAGED(LBM_F32)
