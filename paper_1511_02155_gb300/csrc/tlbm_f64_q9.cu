// tlbm_f64_q9.cu -- D2Q9 kernels of the double storage format
// (see tlbm_ops.cuh).  One translation unit per storage format and lattice.
#include "tlbm_ops.cuh"

TLBM_DEFINE_OPS(ops_fp64_q9, double, 9)
