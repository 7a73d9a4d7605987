// Step kernels for stencil radius 5 (space order 10).
#include "fd_stencil.cuh"
FDGB_INSTANTIATE_RADIUS(5)
