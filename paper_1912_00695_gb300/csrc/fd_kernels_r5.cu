// Step kernels for stencil radius 5 (space order 10).
#include "fd_stencil.cuh"
#include "fd_tma.cuh"
#include "fd_flow.cuh"
FDGB_INSTANTIATE_RADIUS(5)
FDGB_INSTANTIATE_TMA_RADIUS(5)
FDGB_INSTANTIATE_FLOW_RADIUS(5)
