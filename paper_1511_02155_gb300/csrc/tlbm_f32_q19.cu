// tlbm_f32_q19.cu -- D3Q19 kernels of the float storage format
// (see tlbm_ops.cuh).  One translation unit per storage format and lattice.
#include "tlbm_ops.cuh"

TLBM_DEFINE_OPS(ops_fp32_q19, float, 19)
