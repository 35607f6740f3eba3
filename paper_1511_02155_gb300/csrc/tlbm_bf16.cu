// tlbm_bf16.cu -- kernels of the bfloat16 offset storage format, computed in
// float (see tlbm_ops.cuh).
#include "tlbm_ops.cuh"

TLBM_DEFINE_OPS(ops_bf16, __nv_bfloat16)
