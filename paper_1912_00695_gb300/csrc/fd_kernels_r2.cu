// Step kernels for stencil radius 2 (space order 4).
#include "fd_stencil.cuh"
#include "fd_tma.cuh"
#include "fd_flow.cuh"
#include "fd_tma2.cuh"
FDGB_INSTANTIATE_RADIUS(2)
FDGB_INSTANTIATE_TMA_RADIUS(2)
FDGB_INSTANTIATE_TMA2_RADIUS(2)
FDGB_INSTANTIATE_FLOW_RADIUS(2)
