// tlbm_f64.cu -- kernels of the double storage format (see tlbm_ops.cuh).
#include "tlbm_ops.cuh"

TLBM_DEFINE_OPS(ops_fp64, double)
