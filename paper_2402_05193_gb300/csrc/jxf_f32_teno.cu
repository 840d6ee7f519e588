// TENO6-A face sweeps, storage type float: single-phase without viscous
// fluxes and the five-equation model (each viscous order has a unit of its
// own).
#include "jxf_flux_launch.cuh"
JXF_INSTANTIATE_FLUX(float, JXF_SPM, 0, 2)
JXF_INSTANTIATE_FLUX(float, JXF_DIM, 0, 2)
