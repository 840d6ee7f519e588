// Instantiation of the solver kernels for storage type double, model JXF_DIM.
#include "jxf_ops.cuh"
JXF_DEFINE_OPS(ops_f64_dim, double, JXF_DIM)
