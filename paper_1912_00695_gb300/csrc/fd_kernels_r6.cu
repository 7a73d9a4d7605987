// Step kernels for stencil radius 6 (space order 12).
#include "fd_stencil.cuh"
FDGB_INSTANTIATE_RADIUS(6)
