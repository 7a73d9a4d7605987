// Radius dispatch and the small utility kernels around the step kernels:
// extra-source injection, 16-bit level unpacking for read-back and scale
// initialisation.
#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include <atomic>
#include <type_traits>

#include "fd_internal.h"
#include "fd_stencil.cuh"
#include "fd_flow.h"
#include "fd_launch_count.h"

namespace fdgb {

namespace {
std::atomic<long long> g_launches{0};
thread_local long long t_captured = 0;
}  // namespace

cudaError_t counted(cudaError_t e, cudaStream_t s, int n) {
    if (e != cudaSuccess) return e;
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    if (cudaStreamIsCapturing(s, &cs) == cudaSuccess && cs == cudaStreamCaptureStatusActive)
        t_captured += n;
    else
        g_launches.fetch_add(n, std::memory_order_relaxed);
    return e;
}

long long captured_launches() { return t_captured; }

void count_replay(long long n) { g_launches.fetch_add(n, std::memory_order_relaxed); }

long long kernel_launches() { return g_launches.load(std::memory_order_relaxed); }

#define FDGB_DECLARE_RADIUS(R)                                                                   \
    cudaError_t stream_step_radius_##R(int form, int storage, int tile_y, const StepArgs &a,    \
                                       bool check, cudaStream_t s);                             \
    cudaError_t naive_step_radius_##R(int form, int storage, const StepArgs &a, bool check,      \
                                      cudaStream_t s);
FDGB_DECLARE_RADIUS(1)
FDGB_DECLARE_RADIUS(2)
FDGB_DECLARE_RADIUS(3)
FDGB_DECLARE_RADIUS(4)
FDGB_DECLARE_RADIUS(5)
FDGB_DECLARE_RADIUS(6)
FDGB_DECLARE_RADIUS(7)
FDGB_DECLARE_RADIUS(8)
FDGB_DECLARE_RADIUS(9)
FDGB_DECLARE_RADIUS(10)
FDGB_DECLARE_RADIUS(11)
FDGB_DECLARE_RADIUS(12)
#undef FDGB_DECLARE_RADIUS

static cudaError_t launch_stream_step_dispatch(int radius, int form, int storage, int tile_y, const StepArgs &a,
                               bool check, cudaStream_t s) {
    switch (radius) {
        case 1: return stream_step_radius_1(form, storage, tile_y, a, check, s);
        case 2: return stream_step_radius_2(form, storage, tile_y, a, check, s);
        case 3: return stream_step_radius_3(form, storage, tile_y, a, check, s);
        case 4: return stream_step_radius_4(form, storage, tile_y, a, check, s);
        case 5: return stream_step_radius_5(form, storage, tile_y, a, check, s);
        case 6: return stream_step_radius_6(form, storage, tile_y, a, check, s);
        case 7: return stream_step_radius_7(form, storage, tile_y, a, check, s);
        case 8: return stream_step_radius_8(form, storage, tile_y, a, check, s);
        case 9: return stream_step_radius_9(form, storage, tile_y, a, check, s);
        case 10: return stream_step_radius_10(form, storage, tile_y, a, check, s);
        case 11: return stream_step_radius_11(form, storage, tile_y, a, check, s);
        case 12: return stream_step_radius_12(form, storage, tile_y, a, check, s);
        default: return cudaErrorInvalidValue;
    }
}

cudaError_t launch_stream_step(int radius, int form, int storage, int tile_y, const StepArgs &a,
                               bool check, cudaStream_t s) {
    return counted(launch_stream_step_dispatch(radius, form, storage, tile_y, a, check, s), s);
}

static cudaError_t launch_naive_step_dispatch(int radius, int form, int storage, const StepArgs &a, bool check,
                              cudaStream_t s) {
    switch (radius) {
        case 1: return naive_step_radius_1(form, storage, a, check, s);
        case 2: return naive_step_radius_2(form, storage, a, check, s);
        case 3: return naive_step_radius_3(form, storage, a, check, s);
        case 4: return naive_step_radius_4(form, storage, a, check, s);
        case 5: return naive_step_radius_5(form, storage, a, check, s);
        case 6: return naive_step_radius_6(form, storage, a, check, s);
        case 7: return naive_step_radius_7(form, storage, a, check, s);
        case 8: return naive_step_radius_8(form, storage, a, check, s);
        case 9: return naive_step_radius_9(form, storage, a, check, s);
        case 10: return naive_step_radius_10(form, storage, a, check, s);
        case 11: return naive_step_radius_11(form, storage, a, check, s);
        case 12: return naive_step_radius_12(form, storage, a, check, s);
        default: return cudaErrorInvalidValue;
    }
}

cudaError_t launch_naive_step(int radius, int form, int storage, const StepArgs &a, bool check,
                              cudaStream_t s) {
    return counted(launch_naive_step_dispatch(radius, form, storage, a, check, s), s);
}

int stream_grid_x_chunks(int Nx, int x_block) { return (Nx + x_block - 1) / x_block; }

#define FDGB_DECLARE_TMA_RADIUS(R)                                                               \
    cudaError_t tma_step_radius_##R(int form, int storage, int tile_z, int tile_y, int rows,     \
                                    const TmaMaps &map, const StepArgs &a, bool check,           \
                                    cudaStream_t s);                                             \
    bool tma_box_radius_##R(int form, int storage, int tile_z, int tile_y, int rows, int *w, int *h, int *rz);
FDGB_DECLARE_TMA_RADIUS(1)
FDGB_DECLARE_TMA_RADIUS(2)
FDGB_DECLARE_TMA_RADIUS(3)
FDGB_DECLARE_TMA_RADIUS(4)
FDGB_DECLARE_TMA_RADIUS(5)
FDGB_DECLARE_TMA_RADIUS(6)
FDGB_DECLARE_TMA_RADIUS(7)
FDGB_DECLARE_TMA_RADIUS(8)
FDGB_DECLARE_TMA_RADIUS(9)
FDGB_DECLARE_TMA_RADIUS(10)
FDGB_DECLARE_TMA_RADIUS(11)
FDGB_DECLARE_TMA_RADIUS(12)
#undef FDGB_DECLARE_TMA_RADIUS

#define FDGB_DECLARE_BATCH_RADIUS(R)                                                             \
    cudaError_t tma_batch_step_radius_##R(int form, int storage, int tile_z, int tile_y,         \
                                          const BatchShot *shots, const int4 *items, int n_items, \
                                          int offset, cudaStream_t s);
FDGB_DECLARE_BATCH_RADIUS(1)
FDGB_DECLARE_BATCH_RADIUS(2)
FDGB_DECLARE_BATCH_RADIUS(3)
FDGB_DECLARE_BATCH_RADIUS(4)
FDGB_DECLARE_BATCH_RADIUS(5)
FDGB_DECLARE_BATCH_RADIUS(6)
FDGB_DECLARE_BATCH_RADIUS(7)
FDGB_DECLARE_BATCH_RADIUS(8)
FDGB_DECLARE_BATCH_RADIUS(9)
FDGB_DECLARE_BATCH_RADIUS(10)
FDGB_DECLARE_BATCH_RADIUS(11)
FDGB_DECLARE_BATCH_RADIUS(12)
#undef FDGB_DECLARE_BATCH_RADIUS

static cudaError_t launch_tma_batch_step_dispatch(int radius, int form, int storage, int tile_z, int tile_y,
                                  const BatchShot *shots, const int4 *items, int n_items, int offset,
                                  cudaStream_t s) {
    switch (radius) {
#define FDGB_BATCH_R(R) \
        case R: return tma_batch_step_radius_##R(form, storage, tile_z, tile_y, shots, items, n_items, offset, s);
        FDGB_BATCH_R(1) FDGB_BATCH_R(2) FDGB_BATCH_R(3) FDGB_BATCH_R(4)
        FDGB_BATCH_R(5) FDGB_BATCH_R(6) FDGB_BATCH_R(7) FDGB_BATCH_R(8)
        FDGB_BATCH_R(9) FDGB_BATCH_R(10) FDGB_BATCH_R(11) FDGB_BATCH_R(12)
#undef FDGB_BATCH_R
        default: return cudaErrorInvalidValue;
    }
}

cudaError_t launch_tma_batch_step(int radius, int form, int storage, int tile_z, int tile_y,
                                  const BatchShot *shots, const int4 *items, int n_items, int offset,
                                  cudaStream_t s) {
    return counted(launch_tma_batch_step_dispatch(radius, form, storage, tile_z, tile_y, shots, items, n_items, offset, s), s);
}

#define FDGB_DECLARE_GRAD_RADIUS(R)                                                              \
    cudaError_t tma_grad_step_radius_##R(int mode, const TmaMaps &map, const GradMaps &gm,          \
                                         const StepArgs &a, bool check, cudaStream_t s);
FDGB_DECLARE_GRAD_RADIUS(1)
FDGB_DECLARE_GRAD_RADIUS(2)
FDGB_DECLARE_GRAD_RADIUS(3)
FDGB_DECLARE_GRAD_RADIUS(4)
FDGB_DECLARE_GRAD_RADIUS(5)
FDGB_DECLARE_GRAD_RADIUS(6)
FDGB_DECLARE_GRAD_RADIUS(7)
FDGB_DECLARE_GRAD_RADIUS(8)
FDGB_DECLARE_GRAD_RADIUS(9)
FDGB_DECLARE_GRAD_RADIUS(10)
FDGB_DECLARE_GRAD_RADIUS(11)
FDGB_DECLARE_GRAD_RADIUS(12)
#undef FDGB_DECLARE_GRAD_RADIUS

static cudaError_t launch_tma_grad_step_dispatch(int radius, int mode, const TmaMaps &map, const GradMaps &gm, const StepArgs &a,
                                 bool check, cudaStream_t s) {
    switch (radius) {
#define FDGB_GRAD_R(R) \
        case R: return tma_grad_step_radius_##R(mode, map, gm, a, check, s);
        FDGB_GRAD_R(1) FDGB_GRAD_R(2) FDGB_GRAD_R(3) FDGB_GRAD_R(4)
        FDGB_GRAD_R(5) FDGB_GRAD_R(6) FDGB_GRAD_R(7) FDGB_GRAD_R(8)
        FDGB_GRAD_R(9) FDGB_GRAD_R(10) FDGB_GRAD_R(11) FDGB_GRAD_R(12)
#undef FDGB_GRAD_R
        default: return cudaErrorInvalidValue;
    }
}

cudaError_t launch_tma_grad_step(int radius, int mode, const TmaMaps &map, const GradMaps &gm, const StepArgs &a,
                                 bool check, cudaStream_t s) {
    return counted(launch_tma_grad_step_dispatch(radius, mode, map, gm, a, check, s), s);
}

#define FDGB_DECLARE_TMA2_RADIUS(R)                                                              \
    cudaError_t tma2_step_radius_##R(const TmaMaps &map, const StepArgs &a, float *out1, float *out2, \
                                     bool check, cudaStream_t s);                                 \
    void tma2_geometry_radius_##R(int *tz, int *ty, int *box_w, int *box_h, int *ez, int *ey);
FDGB_DECLARE_TMA2_RADIUS(1)
FDGB_DECLARE_TMA2_RADIUS(2)
#undef FDGB_DECLARE_TMA2_RADIUS

static cudaError_t launch_tma2_step_dispatch(int radius, const TmaMaps &map, const StepArgs &a, float *out1, float *out2, bool check,
                             cudaStream_t s) {
    if (radius == 1) return tma2_step_radius_1(map, a, out1, out2, check, s);
    if (radius == 2) return tma2_step_radius_2(map, a, out1, out2, check, s);
    return cudaErrorInvalidValue;
}

cudaError_t launch_tma2_step(int radius, const TmaMaps &map, const StepArgs &a, float *out1, float *out2, bool check,
                             cudaStream_t s) {
    return counted(launch_tma2_step_dispatch(radius, map, a, out1, out2, check, s), s);
}

#define FDGB_DECLARE_FLOW_RADIUS(R)                                                              \
    cudaError_t tma_flow_radius_##R(int form, int storage, int tile_z, int tile_y, int rows, bool ex,   \
                                    const FlowArgs &f, int ctas, bool check, cudaStream_t s);     \
    int tma_flow_occ_radius_##R(int form, int storage, int tile_z, int tile_y, int rows, bool ex); \
    cudaError_t tma_batch_flow_radius_##R(int form, int tile_z, int tile_y, const BatchFlowArgs &f, int ctas, \
                                          cudaStream_t s);                                       \
    int tma_batch_flow_occ_radius_##R(int form, int tile_z, int tile_y);
FDGB_DECLARE_FLOW_RADIUS(1)
FDGB_DECLARE_FLOW_RADIUS(2)
FDGB_DECLARE_FLOW_RADIUS(3)
FDGB_DECLARE_FLOW_RADIUS(4)
FDGB_DECLARE_FLOW_RADIUS(5)
FDGB_DECLARE_FLOW_RADIUS(6)
FDGB_DECLARE_FLOW_RADIUS(7)
FDGB_DECLARE_FLOW_RADIUS(8)
FDGB_DECLARE_FLOW_RADIUS(9)
FDGB_DECLARE_FLOW_RADIUS(10)
FDGB_DECLARE_FLOW_RADIUS(11)
FDGB_DECLARE_FLOW_RADIUS(12)
#undef FDGB_DECLARE_FLOW_RADIUS

static cudaError_t launch_tma_flow_dispatch(int radius, int form, int storage, int tile_z, int tile_y, int rows,
                                            const FlowArgs &f, int ctas, bool check, cudaStream_t s) {
    // receivers or extra sources: the variant that handles them per item
    const bool ex = f.rec_start != nullptr || f.xs_start != nullptr;
    switch (radius) {
#define FDGB_FLOW_R(R) \
        case R: return tma_flow_radius_##R(form, storage, tile_z, tile_y, rows, ex, f, ctas, check, s);
        FDGB_FLOW_R(1) FDGB_FLOW_R(2) FDGB_FLOW_R(3) FDGB_FLOW_R(4)
        FDGB_FLOW_R(5) FDGB_FLOW_R(6) FDGB_FLOW_R(7) FDGB_FLOW_R(8)
        FDGB_FLOW_R(9) FDGB_FLOW_R(10) FDGB_FLOW_R(11) FDGB_FLOW_R(12)
#undef FDGB_FLOW_R
        default: return cudaErrorInvalidValue;
    }
}

cudaError_t launch_tma_flow(int radius, int form, int storage, int tile_z, int tile_y, int rows, const FlowArgs &f,
                            int ctas, bool check, cudaStream_t s) {
    return counted(launch_tma_flow_dispatch(radius, form, storage, tile_z, tile_y, rows, f, ctas, check, s), s);
}

int tma_flow_ctas_per_sm(int radius, int form, int storage, int tile_z, int tile_y, int rows, bool ex) {
    switch (radius) {
#define FDGB_FLOW_O(R) \
        case R: return tma_flow_occ_radius_##R(form, storage, tile_z, tile_y, rows, ex);
        FDGB_FLOW_O(1) FDGB_FLOW_O(2) FDGB_FLOW_O(3) FDGB_FLOW_O(4)
        FDGB_FLOW_O(5) FDGB_FLOW_O(6) FDGB_FLOW_O(7) FDGB_FLOW_O(8)
        FDGB_FLOW_O(9) FDGB_FLOW_O(10) FDGB_FLOW_O(11) FDGB_FLOW_O(12)
#undef FDGB_FLOW_O
        default: return 0;
    }
}

static cudaError_t launch_tma_batch_flow_dispatch(int radius, int form, int tile_z, int tile_y,
                                                  const BatchFlowArgs &f, int ctas, cudaStream_t s) {
    switch (radius) {
#define FDGB_BFLOW_R(R) \
        case R: return tma_batch_flow_radius_##R(form, tile_z, tile_y, f, ctas, s);
        FDGB_BFLOW_R(1) FDGB_BFLOW_R(2) FDGB_BFLOW_R(3) FDGB_BFLOW_R(4)
        FDGB_BFLOW_R(5) FDGB_BFLOW_R(6) FDGB_BFLOW_R(7) FDGB_BFLOW_R(8)
#undef FDGB_BFLOW_R
        default: return cudaErrorInvalidValue;
    }
}

cudaError_t launch_tma_batch_flow(int radius, int form, int tile_z, int tile_y, const BatchFlowArgs &f, int ctas,
                                  cudaStream_t s) {
    return counted(launch_tma_batch_flow_dispatch(radius, form, tile_z, tile_y, f, ctas, s), s);
}

int tma_batch_flow_ctas_per_sm(int radius, int form, int tile_z, int tile_y) {
    switch (radius) {
#define FDGB_BFLOW_O(R) \
        case R: return tma_batch_flow_occ_radius_##R(form, tile_z, tile_y);
        FDGB_BFLOW_O(1) FDGB_BFLOW_O(2) FDGB_BFLOW_O(3) FDGB_BFLOW_O(4)
        FDGB_BFLOW_O(5) FDGB_BFLOW_O(6) FDGB_BFLOW_O(7) FDGB_BFLOW_O(8)
#undef FDGB_BFLOW_O
        default: return 0;
    }
}

bool tma2_geometry(int radius, int *tz, int *ty, int *box_w, int *box_h, int *ez, int *ey) {
    if (radius == 1) tma2_geometry_radius_1(tz, ty, box_w, box_h, ez, ey);
    else if (radius == 2) tma2_geometry_radius_2(tz, ty, box_w, box_h, ez, ey);
    else return false;
    return true;
}

static cudaError_t launch_tma_step_dispatch(int radius, int form, int storage, int tile_z, int tile_y, int rows,
                            const TmaMaps &map, const StepArgs &a, bool check, cudaStream_t s) {
    switch (radius) {
#define FDGB_TMA_R(R) \
        case R: return tma_step_radius_##R(form, storage, tile_z, tile_y, rows, map, a, check, s);
        FDGB_TMA_R(1) FDGB_TMA_R(2) FDGB_TMA_R(3) FDGB_TMA_R(4)
        FDGB_TMA_R(5) FDGB_TMA_R(6) FDGB_TMA_R(7) FDGB_TMA_R(8)
        FDGB_TMA_R(9) FDGB_TMA_R(10) FDGB_TMA_R(11) FDGB_TMA_R(12)
#undef FDGB_TMA_R
        default: return cudaErrorInvalidValue;
    }
}

cudaError_t launch_tma_step(int radius, int form, int storage, int tile_z, int tile_y, int rows,
                            const TmaMaps &map, const StepArgs &a, bool check, cudaStream_t s) {
    return counted(launch_tma_step_dispatch(radius, form, storage, tile_z, tile_y, rows, map, a, check, s), s);
}

bool tma_box(int radius, int form, int storage, int tile_z, int tile_y, int rows, int *w, int *h, int *rz) {
    switch (radius) {
#define FDGB_TMA_B(R) \
        case R: return tma_box_radius_##R(form, storage, tile_z, tile_y, rows, w, h, rz);
        FDGB_TMA_B(1) FDGB_TMA_B(2) FDGB_TMA_B(3) FDGB_TMA_B(4)
        FDGB_TMA_B(5) FDGB_TMA_B(6) FDGB_TMA_B(7) FDGB_TMA_B(8)
        FDGB_TMA_B(9) FDGB_TMA_B(10) FDGB_TMA_B(11) FDGB_TMA_B(12)
#undef FDGB_TMA_B
        default: return false;
    }
}

namespace {

__device__ __forceinline__ int slot_of(long long n) { return int(((n % 3) + 3) % 3); }

template <typename T> __device__ __forceinline__ float to_f(T v);
template <> __device__ __forceinline__ float to_f<float>(float v) { return v; }
template <> __device__ __forceinline__ float to_f<__nv_bfloat16>(__nv_bfloat16 v) {
    return __bfloat162float(v);
}
template <> __device__ __forceinline__ float to_f<__half>(__half v) { return __half2float(v); }
template <typename T> __device__ __forceinline__ T from_f(float v);
template <> __device__ __forceinline__ float from_f<float>(float v) { return v; }
template <> __device__ __forceinline__ __nv_bfloat16 from_f<__nv_bfloat16>(float v) {
    return __float2bfloat16_rn(v);
}
template <> __device__ __forceinline__ __half from_f<__half>(float v) { return __float2half_rn(v); }

// Sources beyond the ones fused into the step kernel, added after the step in
// one thread (in order, so duplicates of a node add up deterministically). The
// step kernel already wrote level n+1 with the scales of slot n+1; 16-bit shots
// add the source to both the increment d^{n+1} and u^{n+1} = u^n + d^{n+1}.
template <typename T>
__global__ void inject_extra_kernel(const StepArgs a, const int *sx, const int *sy, const int *sz,
                                    int first, int count, int expanded, int distinct, float *hist) {
    // distinct nodes: one thread per source (no two threads touch one point);
    // otherwise one thread adds them all in order
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (distinct ? t >= count : t != 0) return;
    if (a.step < 0 || a.step >= a.ld) return;
    T *up = static_cast<T *>(a.up);
    T *un = static_cast<T *>(a.un);
    const int n1 = slot_of(a.step + 1);
    const float s_u = a.scales ? a.scales->scale[n1] : 1.0f;
    const float s_d = a.scales ? a.scales->dscale[n1] : 1.0f;
    const int i0 = distinct ? first + t : first, i1 = distinct ? first + t + 1 : first + count;
    for (int i = i0; i < i1; ++i) {
        const long long p = (long long)sx[i] * a.plane + (long long)sy[i] * a.pz + sz[i];
        const float q = a.wavelet[(long long)i * a.ld + a.step];
        const float w = extra_source_weight(a, p, expanded != 0);
        if constexpr (std::is_same<T, float>::value) {
            add_extra_source_f32(up, p, w, q);
            if (hist) add_extra_source_f32(hist, p, w, q);  // the stored second time difference includes it
        } else {
            up[p] = from_f<T>((to_f<T>(up[p]) * s_d + w * q) / s_d);
            un[p] = from_f<T>((to_f<T>(un[p]) * s_u + w * q) / s_u);
        }
    }
}

// Adjoint sources of the FWI gradient: receiver residuals r^t spread onto
// their nodes (the transpose of the trilinear sampling), gathered per node in a
// fixed order (CSR: node i takes entries row[i]..row[i+1]); the node gets
// w += inc = (dt^2/A) (R^T r)/dt^2 and the gradient its share -inc * D.
__global__ void adjoint_inject_kernel(float *w, float *grad, const float *dhist, const float *f1,
                                      const long long *node_off, const int *row, const int *rec_idx,
                                      const float *rec_w, const float *resid, int nt, int t, float inv_dt2,
                                      int n_nodes) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n_nodes) return;
    float s = 0.0f;
    for (int e = row[i]; e < row[i + 1]; ++e) s = fmaf(rec_w[e], resid[(long long)rec_idx[e] * nt + t], s);
    const long long p = node_off[i];
    const float inc = f1[p] * (s * inv_dt2);
    w[p] += inc;
    grad[p] = fmaf(-inc, dhist[p], grad[p]);
}

// Receivers: trilinear interpolation of the new level u^{n+1} (stored values
// times the level's scale) at each receiver, one thread per receiver, the 8
// corner terms summed in a fixed order (deterministic). off/w: 8 per receiver.
template <typename T>
__global__ void sample_receivers_kernel(const T *u, const LevelScales *scales, int slot, const long long *off,
                                        const float *w, int n, float *out, int stride) {
    const int r = blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= n) return;
    float v = 0.0f;
#pragma unroll
    for (int c = 0; c < 8; ++c) v = fmaf(w[8 * r + c], to_f<T>(u[off[8 * r + c]]), v);
    out[(long long)r * stride] = scales ? v * scales->scale[slot] : v;
}

// Pitched storage-type level -> dense FP32 [Nx][Ny][Nz], times the level scale.
template <typename T>
__global__ void unpack_kernel(const T *src, float *dst, int Nx, int Ny, int Nz, int pz,
                              const LevelScales *scales, int slot) {
    const float s = scales ? scales->scale[slot] : 1.0f;
    const long long n = (long long)Nx * Ny * Nz;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x) {
        const long long z = i % Nz;
        const long long xy = i / Nz;
        dst[i] = to_f<T>(src[xy * pz + z]) * s;
    }
}

// Dense FP32 [Nx][Ny][Nz] -> pitched storage-type level, times 1/scale.
template <typename T>
__global__ void pack_kernel(const float *src, T *dst, int Nx, int Ny, int Nz, int pz, float inv_scale) {
    const long long n = (long long)Nx * Ny * Nz;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x) {
        const long long z = i % Nz;
        const long long xy = i / Nz;
        dst[xy * pz + z] = from_f<T>(src[i] * inv_scale);
    }
}

// u^{n-1} = u^n * s_u - d^n * s_d of a 16-bit shot, pitched -> dense FP32.
template <typename T>
__global__ void unpack_prev_kernel(const T *u, const T *d, float *dst, int Nx, int Ny, int Nz, int pz,
                                   const LevelScales *scales, int slot) {
    const float su = scales->scale[slot], sd = scales->dscale[slot];
    const long long n = (long long)Nx * Ny * Nz;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x) {
        const long long z = i % Nz;
        const long long xy = i / Nz;
        dst[i] = to_f<T>(u[xy * pz + z]) * su - to_f<T>(d[xy * pz + z]) * sd;
    }
}

__global__ void set_level_scale_kernel(LevelScales *ls, int slot, float scale, unsigned amax_bits,
                                       float dscale, unsigned damax_bits) {
    if (threadIdx.x == 0) {
        ls->scale[slot] = scale;
        ls->amax_bits[slot] = amax_bits;
        ls->dscale[slot] = dscale;
        ls->damax_bits[slot] = damax_bits;
    }
}

// The level a BF16 flow launch ended on: unit scales, the launch's maxima.
__global__ void flow_finish_scales_kernel(LevelScales *ls, int slot, const unsigned *amax) {
    if (threadIdx.x == 0) {
        ls->scale[slot] = 1.0f;
        ls->dscale[slot] = 1.0f;
        ls->amax_bits[slot] = amax[0];
        ls->damax_bits[slot] = amax[1];
    }
}

__global__ void init_scales_kernel(LevelScales *ls) {
    if (threadIdx.x < 3) {
        ls->scale[threadIdx.x] = 1.0f;
        ls->amax_bits[threadIdx.x] = 0u;
        ls->dscale[threadIdx.x] = 1.0f;
        ls->damax_bits[threadIdx.x] = 0u;
    }
}

// One pass over the model: validation flags, min(m), and whether eta vanishes
// inside the interior box [nbl, N - nbl)^3 (the kernels then skip its loads there).
__global__ void model_check_kernel(const float *m, const float *eta, int Nx, int Ny, int Nz, int pz, int nbl,
                                   int x_off, int Nx_glob, ModelCheck *out) {
    const long long n = (long long)Nx * Ny * Nz;
    unsigned bad_m = 0, bad_eta = 0, inner = 0, mn = 0x7f800000u;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x) {
        const int z = int(i % Nz);
        const long long xy = i / Nz;
        const int y = int(xy % Ny), x = int(xy / Ny);
        const long long p = xy * pz + z;
        const float mv = m[p];
        if (!(mv > 0.0f) || !isfinite(mv)) bad_m = 1;
        else mn = min(mn, __float_as_uint(mv));
        if (eta) {
            const float e = eta[p];
            if (!(e >= 0.0f) || !isfinite(e)) bad_eta = 1;
            const int xg = x + x_off;  // global plane
            if (e != 0.0f && xg >= nbl && xg < Nx_glob - nbl && y >= nbl && y < Ny - nbl && z >= nbl &&
                z < Nz - nbl)
                inner = 1;
        }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        bad_m |= __shfl_xor_sync(0xffffffffu, bad_m, o);
        bad_eta |= __shfl_xor_sync(0xffffffffu, bad_eta, o);
        inner |= __shfl_xor_sync(0xffffffffu, inner, o);
        mn = min(mn, __shfl_xor_sync(0xffffffffu, mn, o));
    }
    if ((threadIdx.x & 31) == 0) {
        if (bad_m) atomicOr(&out->bad_m, 1u);
        if (bad_eta) atomicOr(&out->bad_eta, 1u);
        if (inner) atomicOr(&out->eta_interior_nonzero, 1u);
        atomicMin(&out->min_m_bits, mn);
    }
}

// eta = m * d_max * sum_a (l_a / nbl)^2, l_a the depth into the layer along axis a.
__global__ void default_damping_kernel(const float *m, float *eta, int Nx, int Ny, int Nz, int pz, int nbl,
                                       float dmax) {
    const long long n = (long long)Nx * Ny * Nz;
    const float inv = nbl > 0 ? 1.0f / float(nbl) : 0.0f;
    auto frac2 = [&](int i, int N) {
        const int d = max(max(nbl - i, i - (N - 1 - nbl)), 0);
        const float f = float(d) * inv;
        return f * f;
    };
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x) {
        const int z = int(i % Nz);
        const long long xy = i / Nz;
        const int y = int(xy % Ny), x = int(xy / Ny);
        const long long p = xy * pz + z;
        eta[p] = nbl > 0 ? m[p] * (dmax * (frac2(x, Nx) + frac2(y, Ny) + frac2(z, Nz))) : 0.0f;
    }
}

// Factored form's per-point coefficients, in place: (m, eta) -> (w, g) with
// w = dt^2 / (m + dt/2 eta), g = (dt/2 eta) / (m + dt/2 eta) (correctly rounded
// divisions; padding elements are zero in both and stay zero).
__global__ void prepare_factored_kernel(float *f1, float *f2, long long n, float half_dt, float dt2) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x) {
        const float mv = f1[i], he = half_dt * f2[i];
        const float r0 = mv + he;
        if (r0 > 0.0f) {
            f1[i] = __fdiv_rn(dt2, r0);
            f2[i] = __fdiv_rn(he, r0);
        }
    }
}

}  // namespace

cudaError_t launch_model_check(const float *m, const float *eta, int Nx, int Ny, int Nz, int pz, int nbl,
                               int x_off, int Nx_glob, ModelCheck *out, cudaStream_t s) {
    model_check_kernel<<<1216, 256, 0, s>>>(m, eta, Nx, Ny, Nz, pz, nbl, x_off, Nx_glob, out);
    return counted(cudaGetLastError(), s);
}

cudaError_t launch_default_damping(const float *m, float *eta, int Nx, int Ny, int Nz, int pz, int nbl,
                                   float dmax, cudaStream_t s) {
    default_damping_kernel<<<1216, 256, 0, s>>>(m, eta, Nx, Ny, Nz, pz, nbl, dmax);
    return counted(cudaGetLastError(), s);
}

cudaError_t launch_prepare_factored(float *f1, float *f2, long long n_pitched, float half_dt, float dt2,
                                    cudaStream_t s) {
    prepare_factored_kernel<<<1216, 256, 0, s>>>(f1, f2, n_pitched, half_dt, dt2);
    return counted(cudaGetLastError(), s);
}

cudaError_t launch_inject_extra(const StepArgs &a, const int *sx, const int *sy, const int *sz,
                                int first, int count, int storage, int expanded, bool distinct, cudaStream_t s,
                                float *hist) {
    if (count <= 0) return cudaSuccess;
    const int threads = 64, blocks = distinct ? (count + threads - 1) / threads : 1;
    const int d = distinct ? 1 : 0;
    if (storage == kF32)
        inject_extra_kernel<float><<<blocks, threads, 0, s>>>(a, sx, sy, sz, first, count, expanded, d, hist);
    else if (storage == kBF16)
        inject_extra_kernel<__nv_bfloat16><<<blocks, threads, 0, s>>>(a, sx, sy, sz, first, count, expanded, d,
                                                                      nullptr);
    else if (storage == kF16)
        inject_extra_kernel<__half><<<blocks, threads, 0, s>>>(a, sx, sy, sz, first, count, expanded, d, nullptr);
    else return cudaErrorInvalidValue;
    return counted(cudaGetLastError(), s);
}

cudaError_t launch_adjoint_inject(float *w, float *grad, const float *dhist, const float *f1,
                                  const long long *node_off, const int *row, const int *rec_idx, const float *rec_w,
                                  const float *resid, int nt, int t, float inv_dt2, int n_nodes, cudaStream_t s) {
    if (n_nodes <= 0) return cudaSuccess;
    const int threads = 128, blocks = (n_nodes + threads - 1) / threads;
    adjoint_inject_kernel<<<blocks, threads, 0, s>>>(w, grad, dhist, f1, node_off, row, rec_idx, rec_w, resid, nt, t,
                                                     inv_dt2, n_nodes);
    return counted(cudaGetLastError(), s);
}

__global__ void residual_kernel(const float *syn, float *obs_to_res, long long n) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
        obs_to_res[i] = syn[i] - obs_to_res[i];
}

cudaError_t launch_residual(const float *syn, float *obs_to_res, size_t n, cudaStream_t s) {
    if (n == 0) return cudaSuccess;
    residual_kernel<<<608, 256, 0, s>>>(syn, obs_to_res, (long long)n);
    return counted(cudaGetLastError(), s);
}

cudaError_t launch_sample_receivers(const void *u, int storage, const LevelScales *scales, int slot,
                                    const long long *off, const float *w, int n, float *out, int stride,
                                    cudaStream_t s) {
    if (n <= 0) return cudaSuccess;
    const int threads = 128, blocks = (n + threads - 1) / threads;
    if (storage == kF32)
        sample_receivers_kernel<float><<<blocks, threads, 0, s>>>(static_cast<const float *>(u), nullptr, slot,
                                                                   off, w, n, out, stride);
    else if (storage == kBF16)
        sample_receivers_kernel<__nv_bfloat16><<<blocks, threads, 0, s>>>(
            static_cast<const __nv_bfloat16 *>(u), scales, slot, off, w, n, out, stride);
    else if (storage == kF16)
        sample_receivers_kernel<__half><<<blocks, threads, 0, s>>>(static_cast<const __half *>(u), scales, slot,
                                                                    off, w, n, out, stride);
    else
        return cudaErrorInvalidValue;
    return counted(cudaGetLastError(), s);
}

cudaError_t launch_unpack_level(const void *src, float *dst, int Nx, int Ny, int Nz, int pz,
                                int storage, const LevelScales *scales, int slot, cudaStream_t s) {
    const int blocks = 1024, threads = 256;
    if (storage == kF32)
        unpack_kernel<float><<<blocks, threads, 0, s>>>(static_cast<const float *>(src), dst, Nx, Ny,
                                                        Nz, pz, nullptr, slot);
    else if (storage == kBF16)
        unpack_kernel<__nv_bfloat16><<<blocks, threads, 0, s>>>(
            static_cast<const __nv_bfloat16 *>(src), dst, Nx, Ny, Nz, pz, scales, slot);
    else if (storage == kF16)
        unpack_kernel<__half><<<blocks, threads, 0, s>>>(static_cast<const __half *>(src), dst, Nx, Ny,
                                                         Nz, pz, scales, slot);
    else return cudaErrorInvalidValue;
    return counted(cudaGetLastError(), s);
}

cudaError_t launch_pack_level(const float *src, void *dst, int Nx, int Ny, int Nz, int pz,
                              int storage, float inv_scale, cudaStream_t s) {
    const int blocks = 1024, threads = 256;
    if (storage == kF32)
        pack_kernel<float><<<blocks, threads, 0, s>>>(src, static_cast<float *>(dst), Nx, Ny, Nz, pz, inv_scale);
    else if (storage == kBF16)
        pack_kernel<__nv_bfloat16><<<blocks, threads, 0, s>>>(src, static_cast<__nv_bfloat16 *>(dst), Nx, Ny,
                                                              Nz, pz, inv_scale);
    else if (storage == kF16)
        pack_kernel<__half><<<blocks, threads, 0, s>>>(src, static_cast<__half *>(dst), Nx, Ny, Nz, pz,
                                                       inv_scale);
    else return cudaErrorInvalidValue;
    return counted(cudaGetLastError(), s);
}

cudaError_t launch_flow_finish_scales(LevelScales *scales, int slot, const unsigned *amax, cudaStream_t s) {
    flow_finish_scales_kernel<<<1, 32, 0, s>>>(scales, slot, amax);
    return counted(cudaGetLastError(), s);
}

cudaError_t launch_set_level_scale(LevelScales *scales, int slot, float scale, unsigned amax_bits,
                                   float dscale, unsigned damax_bits, cudaStream_t s) {
    set_level_scale_kernel<<<1, 32, 0, s>>>(scales, slot, scale, amax_bits, dscale, damax_bits);
    return counted(cudaGetLastError(), s);
}

cudaError_t launch_unpack_prev(const void *u, const void *d, float *dst, int Nx, int Ny, int Nz, int pz,
                               int storage, const LevelScales *scales, int slot, cudaStream_t s) {
    const int blocks = 1024, threads = 256;
    if (storage == kBF16)
        unpack_prev_kernel<__nv_bfloat16><<<blocks, threads, 0, s>>>(
            static_cast<const __nv_bfloat16 *>(u), static_cast<const __nv_bfloat16 *>(d), dst, Nx, Ny, Nz, pz,
            scales, slot);
    else if (storage == kF16)
        unpack_prev_kernel<__half><<<blocks, threads, 0, s>>>(static_cast<const __half *>(u),
                                                              static_cast<const __half *>(d), dst, Nx, Ny, Nz,
                                                              pz, scales, slot);
    else return cudaErrorInvalidValue;
    return counted(cudaGetLastError(), s);
}

cudaError_t launch_init_scales(LevelScales *scales, cudaStream_t s) {
    init_scales_kernel<<<1, 32, 0, s>>>(scales);
    return counted(cudaGetLastError(), s);
}

}  // namespace fdgb
