// Step kernels for stencil radius 3 (space order 6).
#include "fd_stencil.cuh"
FDGB_INSTANTIATE_RADIUS(3)
