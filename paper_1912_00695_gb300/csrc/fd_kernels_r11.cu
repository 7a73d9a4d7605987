// Step kernels for stencil radius 11 (space order 22).
#include "fd_stencil.cuh"
#include "fd_tma.cuh"
#include "fd_flow.cuh"
FDGB_INSTANTIATE_RADIUS(11)
FDGB_INSTANTIATE_TMA_RADIUS(11)
FDGB_INSTANTIATE_FLOW_RADIUS(11)
