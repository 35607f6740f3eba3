// tlbm_f16_q9.cu -- D2Q9 kernels of the IEEE-half offset storage format, computed in float
// (see tlbm_ops.cuh).  One translation unit per storage format and lattice.
#include "tlbm_ops.cuh"

TLBM_DEFINE_OPS(ops_fp16_q9, __half, 9)
