// TENO6-A face sweeps with order-2 central viscous fluxes, storage type
// double, single-phase model.
#include "jxf_flux_launch.cuh"
JXF_INSTANTIATE_FLUX(double, JXF_SPM, 1, 2)
