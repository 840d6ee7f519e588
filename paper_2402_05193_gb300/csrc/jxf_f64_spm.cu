// Instantiation of the solver kernels for storage type double, model JXF_SPM.
#include "jxf_ops.cuh"
JXF_DEFINE_OPS(ops_f64_spm, double, JXF_SPM)
