// tlbm_bf16_q9.cu -- D2Q9 kernels of the bfloat16 offset storage format, computed in float
// (see tlbm_ops.cuh).  One translation unit per storage format and lattice.
#include "tlbm_ops.cuh"

TLBM_DEFINE_OPS(ops_bf16_q9, __nv_bfloat16, 9)
