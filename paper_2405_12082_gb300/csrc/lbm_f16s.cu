// lbm_f16s.cu -- kernels for LBM_F16S population storage.
#include "lbm_kernels.cuh"

LBM_INSTANTIATE(LBM_F16S)
