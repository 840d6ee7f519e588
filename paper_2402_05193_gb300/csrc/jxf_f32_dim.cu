// Instantiation of the solver kernels for storage type float, model JXF_DIM.
#include "jxf_ops.cuh"
JXF_DEFINE_OPS(ops_f32_dim, float, JXF_DIM)
