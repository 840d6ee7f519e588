// Instantiation of the solver kernels for storage type double and model JXF_SPM:
// the launch table and the face sweeps without viscous fluxes (each viscous
// order has a unit of its own).
#include "jxf_flux_launch.cuh"
JXF_EXTERN_FLUX(double, JXF_SPM, 1, 0)
JXF_EXTERN_FLUX(double, JXF_SPM, 2, 0)
JXF_EXTERN_FLUX(double, JXF_SPM, 3, 0)
JXF_EXTERN_FLUX(double, JXF_SPM, 0, 2)
JXF_EXTERN_FLUX(double, JXF_SPM, 1, 2)
JXF_EXTERN_FLUX(double, JXF_SPM, 2, 2)
JXF_EXTERN_FLUX(double, JXF_SPM, 3, 2)
JXF_DEFINE_OPS(ops_f64_spm, double, JXF_SPM)
JXF_INSTANTIATE_FLUX(double, JXF_SPM, 0, 0)
