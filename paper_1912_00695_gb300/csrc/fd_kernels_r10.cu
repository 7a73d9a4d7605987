// Step kernels for stencil radius 10 (space order 20).
#include "fd_stencil.cuh"
#include "fd_tma.cuh"
#include "fd_flow.cuh"
FDGB_INSTANTIATE_RADIUS(10)
FDGB_INSTANTIATE_TMA_RADIUS(10)
FDGB_INSTANTIATE_FLOW_RADIUS(10)
