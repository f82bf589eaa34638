// lbm_f64.cu -- kernels for LBM_F64 population storage.
#include "lbm_kernels.cuh"

LBM_INSTANTIATE(LBM_F64)
