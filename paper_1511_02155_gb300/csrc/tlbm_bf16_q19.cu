// tlbm_bf16_q19.cu -- D3Q19 kernels of the bfloat16 offset storage format, computed in float
// (see tlbm_ops.cuh).  One translation unit per storage format and lattice.
#include "tlbm_ops.cuh"

TLBM_DEFINE_OPS(ops_bf16_q19, __nv_bfloat16, 19)
