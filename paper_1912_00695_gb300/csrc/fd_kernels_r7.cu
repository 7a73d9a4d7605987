// Step kernels for stencil radius 7 (space order 14).
#include "fd_stencil.cuh"
FDGB_INSTANTIATE_RADIUS(7)
