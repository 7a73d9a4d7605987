// Step kernels for stencil radius 2 (space order 4).
#include "fd_stencil.cuh"
FDGB_INSTANTIATE_RADIUS(2)
