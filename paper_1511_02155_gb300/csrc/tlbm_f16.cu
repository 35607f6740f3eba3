// tlbm_f16.cu -- kernels of the IEEE-half offset storage format, computed in
// float (see tlbm_ops.cuh).
#include "tlbm_ops.cuh"

TLBM_DEFINE_OPS(ops_fp16, __half)
