// Step kernels for stencil radius 4 (space order 8).
#include "fd_stencil.cuh"
#include "fd_tma.cuh"
#include "fd_flow.cuh"
FDGB_INSTANTIATE_RADIUS(4)
FDGB_INSTANTIATE_TMA_RADIUS(4)
FDGB_INSTANTIATE_FLOW_RADIUS(4)
