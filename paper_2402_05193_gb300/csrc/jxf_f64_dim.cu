// Instantiation of the solver kernels for storage type double and model JXF_DIM:
// the launch table and the face sweeps without viscous fluxes (each viscous
// order has a unit of its own).
#include "jxf_flux_launch.cuh"
JXF_EXTERN_FLUX(double, JXF_DIM, 0, 2)
JXF_DEFINE_OPS(ops_f64_dim, double, JXF_DIM)
JXF_INSTANTIATE_FLUX(double, JXF_DIM, 0, 0)
