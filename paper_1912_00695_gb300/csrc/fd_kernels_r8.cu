// Step kernels for stencil radius 8 (space order 16).
#include "fd_stencil.cuh"
#include "fd_tma.cuh"
#include "fd_flow.cuh"
FDGB_INSTANTIATE_RADIUS(8)
FDGB_INSTANTIATE_TMA_RADIUS(8)
FDGB_INSTANTIATE_FLOW_RADIUS(8)
