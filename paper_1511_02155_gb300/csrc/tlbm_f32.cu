// tlbm_f32.cu -- kernels of the float storage format (see tlbm_ops.cuh).
#include "tlbm_ops.cuh"

TLBM_DEFINE_OPS(ops_fp32, float)
