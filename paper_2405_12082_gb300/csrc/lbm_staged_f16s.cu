// lbm_staged_f16s.cu -- staged step kernels for LBM_F16S population storage.
#include "lbm_staged.cuh"

LBM_INSTANTIATE_STAGED(LBM_F16S)
