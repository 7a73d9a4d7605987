// Step kernels for stencil radius 12 (space order 24).
#include "fd_stencil.cuh"
#include "fd_tma.cuh"
#include "fd_flow.cuh"
FDGB_INSTANTIATE_RADIUS(12)
FDGB_INSTANTIATE_TMA_RADIUS(12)
FDGB_INSTANTIATE_FLOW_RADIUS(12)
