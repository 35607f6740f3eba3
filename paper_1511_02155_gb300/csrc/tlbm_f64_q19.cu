// tlbm_f64_q19.cu -- D3Q19 kernels of the double storage format
// (see tlbm_ops.cuh).  One translation unit per storage format and lattice.
#include "tlbm_ops.cuh"

TLBM_DEFINE_OPS(ops_fp64_q19, double, 19)
