// Face sweeps with order-4 central viscous fluxes, storage type float,
// single-phase model.
#include "jxf_flux_launch.cuh"
JXF_INSTANTIATE_FLUX(float, JXF_SPM, 2, 0)
