// Instantiation of the solver kernels for storage type float, model JXF_SPM.
#include "jxf_ops.cuh"
JXF_DEFINE_OPS(ops_f32_spm, float, JXF_SPM)
