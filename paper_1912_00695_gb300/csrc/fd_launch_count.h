// Count of this library's kernel launches, executed or queued for execution.
// Every launcher reports its launch; a launch recorded into a CUDA graph is
// counted each time the graph is replayed, not when it is recorded.
#pragma once
#include <cuda_runtime.h>

namespace fdgb {

// Passes `e` through; on success counts `n` launches on stream `s` (as recorded
// into this thread's graph if `s` is capturing, else as executed).
cudaError_t counted(cudaError_t e, cudaStream_t s, int n = 1);
// Launches this thread has recorded into graphs so far.
long long captured_launches();
// A replay of a graph holding `n` launches.
void count_replay(long long n);
// Executed or queued launches since the library was loaded (all threads).
long long kernel_launches();

}  // namespace fdgb
