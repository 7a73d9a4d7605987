// Step kernels for stencil radius 6 (space order 12).
#include "fd_stencil.cuh"
#include "fd_tma.cuh"
#include "fd_flow.cuh"
FDGB_INSTANTIATE_RADIUS(6)
FDGB_INSTANTIATE_TMA_RADIUS(6)
FDGB_INSTANTIATE_FLOW_RADIUS(6)
