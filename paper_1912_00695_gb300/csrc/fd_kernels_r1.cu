// Step kernels for stencil radius 1 (space order 2).
#include "fd_stencil.cuh"
FDGB_INSTANTIATE_RADIUS(1)
