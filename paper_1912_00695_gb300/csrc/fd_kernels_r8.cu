// Step kernels for stencil radius 8 (space order 16).
#include "fd_stencil.cuh"
FDGB_INSTANTIATE_RADIUS(8)
