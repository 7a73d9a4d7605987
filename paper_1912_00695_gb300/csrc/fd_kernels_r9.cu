// Step kernels for stencil radius 9 (space order 18).
#include "fd_stencil.cuh"
#include "fd_tma.cuh"
#include "fd_flow.cuh"
FDGB_INSTANTIATE_RADIUS(9)
FDGB_INSTANTIATE_TMA_RADIUS(9)
FDGB_INSTANTIATE_FLOW_RADIUS(9)
