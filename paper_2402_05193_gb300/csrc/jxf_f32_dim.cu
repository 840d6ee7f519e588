// Instantiation of the solver kernels for storage type float and model JXF_DIM:
// the launch table and the face sweeps without viscous fluxes (each viscous
// order has a unit of its own).
#include "jxf_flux_launch.cuh"
JXF_EXTERN_FLUX(float, JXF_DIM, 0, 2)
JXF_DEFINE_OPS(ops_f32_dim, float, JXF_DIM)
JXF_INSTANTIATE_FLUX(float, JXF_DIM, 0, 0)
