// Periodic-boundary step (test mode of the solver): see fd_periodic.cu.
#pragma once
#include <cuda_runtime.h>

#include "fd_internal.h"

namespace fdgb {

// One FP32 step from a.u, a.up to a.up with every tap index wrapped around the
// computational extent (a 3-torus); radius 1..kMaxRadius, either form.
cudaError_t launch_periodic_step(int radius, int form, const StepArgs &a, bool check, cudaStream_t s);

}  // namespace fdgb
