// Self-test of the device-side bounded waits (failure detection without a
// fault): one CTA waits on a ring mbarrier that no copy or thread completes and
// on a dependency flag that nothing sets, with the very wait functions the step
// kernels use; each gives up after its time limit and the kernel returns, so
// the context stays usable and the host reads what happened.
#include "../../include/fd_acoustic.h"
#include "fd_flow.cuh"
#include "fd_launch_count.h"

namespace fdgb {
void set_last_error(const char *msg);  // fd_api.cu: the fd_last_error() text

namespace {

__global__ void selftest_waits_kernel(const unsigned *flag, const unsigned *abort, unsigned long long *out) {
    __shared__ __align__(8) uint64_t bar;
    if (threadIdx.x != 0) return;
    const uint32_t b = smem_addr(&bar);
    mbar_init(b, 1);  // one arrival pending: phase 0 never completes
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    unsigned long long t0 = global_ns();
    const bool mbar_done = mbar_wait_bounded(b, 0);
    unsigned long long t1 = global_ns();
    const bool flag_done = flow_wait(flag, 1u, abort);
    unsigned long long t2 = global_ns();
    out[0] = (mbar_done ? 0u : 1u) | (flag_done ? 0u : 2u);
    out[1] = t1 - t0;
    out[2] = t2 - t1;
}

}  // namespace
}  // namespace fdgb

using namespace fdgb;

extern "C" int fd_selftest_waits(unsigned *status, double *mbar_seconds, double *flag_seconds) {
    if (!status) return FD_EINVAL;
    void *buf = nullptr;
    if (cudaMalloc(&buf, 64) != cudaSuccess) {
        cudaGetLastError();
        return FD_ENOMEM;
    }
    unsigned long long out[3] = {0, 0, 0};
    cudaError_t e = cudaMemset(buf, 0, 64);
    unsigned *flag = static_cast<unsigned *>(buf);
    unsigned *abort_word = flag + 1;
    unsigned long long *res = reinterpret_cast<unsigned long long *>(static_cast<char *>(buf) + 32);
    if (e == cudaSuccess) {
        selftest_waits_kernel<<<1, 32>>>(flag, abort_word, res);
        e = counted(cudaGetLastError(), nullptr);
    }
    if (e == cudaSuccess) e = cudaDeviceSynchronize();
    if (e == cudaSuccess) e = cudaMemcpy(out, res, sizeof out, cudaMemcpyDeviceToHost);
    cudaFree(buf);
    if (e != cudaSuccess) {
        set_last_error(cudaGetErrorString(e));
        return FD_ECUDA;
    }
    *status = unsigned(out[0]);
    if (mbar_seconds) *mbar_seconds = double(out[1]) * 1e-9;
    if (flag_seconds) *flag_seconds = double(out[2]) * 1e-9;
    return FD_OK;
}
