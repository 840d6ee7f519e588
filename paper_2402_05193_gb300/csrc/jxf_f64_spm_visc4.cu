// Face sweeps with order-4 central viscous fluxes, storage type double,
// single-phase model.
#include "jxf_flux_launch.cuh"
JXF_INSTANTIATE_FLUX(double, JXF_SPM, 2, 0)
