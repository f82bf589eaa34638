// lbm_staged_f64.cu -- staged step kernels for LBM_F64 population storage.
#include "lbm_staged.cuh"

LBM_INSTANTIATE_STAGED(LBM_F64)
