// Step kernels for stencil radius 7 (space order 14).
#include "fd_stencil.cuh"
#include "fd_tma.cuh"
#include "fd_flow.cuh"
FDGB_INSTANTIATE_RADIUS(7)
FDGB_INSTANTIATE_TMA_RADIUS(7)
FDGB_INSTANTIATE_FLOW_RADIUS(7)
