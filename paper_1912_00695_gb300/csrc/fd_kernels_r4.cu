// Step kernels for stencil radius 4 (space order 8).
#include "fd_stencil.cuh"
FDGB_INSTANTIATE_RADIUS(4)
