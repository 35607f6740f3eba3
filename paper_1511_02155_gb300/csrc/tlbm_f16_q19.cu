// tlbm_f16_q19.cu -- D3Q19 kernels of the IEEE-half offset storage format, computed in float
// (see tlbm_ops.cuh).  One translation unit per storage format and lattice.
#include "tlbm_ops.cuh"

TLBM_DEFINE_OPS(ops_fp16_q19, __half, 19)
