// Step kernels for stencil radius 3 (space order 6).
#include "fd_stencil.cuh"
#include "fd_tma.cuh"
#include "fd_flow.cuh"
FDGB_INSTANTIATE_RADIUS(3)
FDGB_INSTANTIATE_TMA_RADIUS(3)
FDGB_INSTANTIATE_FLOW_RADIUS(3)
