// lbm_f32.cu -- kernels for LBM_F32 population storage.
#include "lbm_kernels.cuh"

LBM_INSTANTIATE(LBM_F32)
