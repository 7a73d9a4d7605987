// fd_forward_noalloc: time steps on caller-owned device buffers with no device
// allocation at all. The step kernel's scratch (per-CTA maxima of |u| and the
// running maximum over the call) lives in one file-scope __device__ array
// instead of a cudaMalloc'd buffer; the caller passes every input and output.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <utility>

#include "../../include/fd_acoustic.h"
#include "fd_launch_count.h"
#include "fd_stencil.cuh"

// sources this entry point accepts (its documented limit)
constexpr int kNoallocSources = 4;
// space orders this entry point accepts (its documented limit)
constexpr int kNoallocMaxRadius = 8;

namespace fdgb {
void set_last_error(const char *msg);  // fd_api.cu: the fd_last_error() text

namespace {

constexpr int kNoAllocMaxCtas = 16384;  // CTAs one step may launch
constexpr int kNoAllocTY = 8;
constexpr int kNoAllocMaxDevices = 64;

// Scratch: word 0 = running max |u| (float bits) over the call's steps, words
// 64.. = one partial max per CTA of the current step. 65,792 bytes per device,
// held by every GPU that loads the library until the process exits.
static __device__ __align__(256) unsigned g_noalloc_scratch[64 + kNoAllocMaxCtas];

std::mutex g_noalloc_mu;
unsigned *g_noalloc_ptr[kNoAllocMaxDevices] = {};
int g_noalloc_sms[kNoAllocMaxDevices] = {};  // multiprocessors of each device, read with its address

// Streaming step (expanded form, FP32 storage, dense [Nx][Ny][Nz] layout): the
// same per-point arithmetic as fd_stream_kernel<R, kExpanded, TY, float>, with
// the maximum of |u^{n+1}| written as one partial per CTA into the scratch.
template <int R>
__global__ void __launch_bounds__(32 * kNoAllocTY) noalloc_step_kernel(const StepArgs a,
                                                                       unsigned *partials) {
    constexpr int TY = kNoAllocTY;
    constexpr int TZ = kTileZ;
    constexpr int SW = TZ + 2 * R;
    constexpr int SH = TY + 2 * R;
    constexpr int NYH = (R + TY - 1) / TY;
    __shared__ float tile[2][SH][SW];
    __shared__ unsigned warp_max[TY];

    const int tz = threadIdx.x, ty = threadIdx.y;
    const int z0 = blockIdx.x * TZ, y0 = blockIdx.y * TY;
    const int z = z0 + tz, y = y0 + ty;
    const int xb = blockIdx.z * a.x_block;
    const int xe = min(xb + a.x_block, a.Nx);
    const bool own = (y < a.Ny) && (z < a.Nz);
    const float *__restrict__ u = static_cast<const float *>(a.u);
    float *up = static_cast<float *>(a.up);
    const long long P = a.plane;
    const long long col = (long long)y * a.pz + z;
    const bool yz_box = y >= a.by0 && y < a.by1 && z >= a.bz0 && z < a.bz1;

    unsigned src_mask = 0;
    if (own)
        for (int s = 0; s < a.ns && s < kFusedSources; ++s)
            if (a.sy[s] == y && a.sz[s] == z && a.sx[s] >= xb && a.sx[s] < xe) src_mask |= 1u << s;

    float hy_lo[NYH], hy_hi[NYH], hz_lo, hz_hi;
    auto load_halo = [&](int x) {
        const long long px = (long long)x * P;
#pragma unroll
        for (int k = 0; k < NYH; ++k) {
            const int i = ty + k * TY;
            hy_lo[k] = 0.0f;
            hy_hi[k] = 0.0f;
            if (i < R && z < a.Nz) {
                const int ya = y0 - R + i, yb = y0 + TY + i;
                if (ya >= 0) hy_lo[k] = __ldg(u + px + (long long)ya * a.pz + z);
                if (yb < a.Ny) hy_hi[k] = __ldg(u + px + (long long)yb * a.pz + z);
            }
        }
        hz_lo = 0.0f;
        hz_hi = 0.0f;
        if (tz < R && y < a.Ny) {
            const int za = z0 - R + tz, zb = z0 + TZ + tz;
            if (za >= 0) hz_lo = __ldg(u + px + (long long)y * a.pz + za);
            if (zb < a.Nz) hz_hi = __ldg(u + px + (long long)y * a.pz + zb);
        }
    };
    auto store_halo = [&](int buf) {
#pragma unroll
        for (int k = 0; k < NYH; ++k) {
            const int i = ty + k * TY;
            if (i < R) {
                tile[buf][i][tz + R] = hy_lo[k];
                tile[buf][TY + R + i][tz + R] = hy_hi[k];
            }
        }
        if (tz < R) {
            tile[buf][ty + R][tz] = hz_lo;
            tile[buf][ty + R][TZ + R + tz] = hz_hi;
        }
    };
    auto load_u = [&](int x) -> float {
        return (own && x >= 0 && x < a.Nx) ? __ldg(u + (long long)x * P + col) : 0.0f;
    };

    float q[2 * R + 1];
#pragma unroll
    for (int i = 0; i < 2 * R; ++i) q[i] = load_u(xb - R + i);
    float nxt = load_u(xb + R);
    load_halo(xb);
    float pum = 0.0f, pm = 0.0f, pe = 0.0f;
    auto load_point = [&](int x) {
        if (own) {
            const long long p = (long long)x * P + col;
            pum = up[p];
            pm = __ldg(a.f1 + p);
            const bool in_box = yz_box && x >= a.bx0 && x < a.bx1;
            pe = in_box ? 0.0f : __ldg(a.f2 + p);
        }
    };
    load_point(xb);

    unsigned amax_bits = 0;
    for (int x = xb; x < xe; ++x) {
        const int buf = (x - xb) & 1;
        q[2 * R] = nxt;
        store_halo(buf);
        tile[buf][ty + R][tz + R] = q[R];
        __syncthreads();
        const float cum = pum, cm = pm, ce = pe;
        if (x + 1 < xe) {
            load_halo(x + 1);
            nxt = load_u(x + 1 + R);
            load_point(x + 1);
        }
        if (own) {
            const float(*t)[SW] = tile[buf];
            const int cy = ty + R, cz = tz + R;
            const float uc = q[R];
            const float inv = expanded_inv(fmaf(a.half_dt, ce, cm));
            float taps = 0.0f;
#pragma unroll
            for (int j = 1; j <= R; ++j) {
                const float cj = a.coef[j] * inv;
                taps = fmaf(cj, q[R - j] - uc, taps);
                taps = fmaf(cj, q[R + j] - uc, taps);
                taps = fmaf(cj, t[cy - j][cz] - uc, taps);
                taps = fmaf(cj, t[cy + j][cz] - uc, taps);
                taps = fmaf(cj, t[cy][cz - j] - uc, taps);
                taps = fmaf(cj, t[cy][cz + j] - uc, taps);
            }
            float src_w;
            float v = Update<kExpanded>::apply(taps, uc, cum, cm, ce, inv, a, src_w);
            if (src_mask) {
#pragma unroll
                for (int s = 0; s < kFusedSources; ++s)
                    if (((src_mask >> s) & 1u) && a.sx[s] == x) v = fmaf(src_w, source_value(a, s), v);
            }
            up[(long long)x * P + col] = v;
            amax_bits = max(amax_bits, __float_as_uint(fabsf(v)));
        }
#pragma unroll
        for (int i = 0; i < 2 * R; ++i) q[i] = q[i + 1];
    }
    // one partial per CTA: warp maxima through shared memory, then one store
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) amax_bits = max(amax_bits, __shfl_xor_sync(0xffffffffu, amax_bits, o));
    if (tz == 0) warp_max[ty] = amax_bits;
    __syncthreads();
    if (tz == 0 && ty == 0) {
        unsigned mx = 0;
        for (int w = 0; w < TY; ++w) mx = max(mx, warp_max[w]);
        const int cta = blockIdx.x + gridDim.x * (blockIdx.y + gridDim.y * blockIdx.z);
        partials[cta] = mx;
    }
}

// Fold the step's per-CTA partials into the running maximum (word 0).
__global__ void noalloc_reduce_kernel(unsigned *scratch, int n_partials) {
    __shared__ unsigned red[256];
    unsigned mx = 0;
    for (int i = threadIdx.x; i < n_partials; i += blockDim.x) mx = max(mx, scratch[64 + i]);
    red[threadIdx.x] = mx;
    __syncthreads();
    for (int s = blockDim.x / 2; s > 0; s >>= 1) {
        if (threadIdx.x < s) red[threadIdx.x] = max(red[threadIdx.x], red[threadIdx.x + s]);
        __syncthreads();
    }
    if (threadIdx.x == 0) scratch[0] = max(scratch[0], red[0]);
}

__global__ void noalloc_clear_kernel(unsigned *scratch) {
    if (threadIdx.x == 0) scratch[0] = 0u;
}

template <int R>
cudaError_t launch_noalloc(const StepArgs &a, dim3 grid, unsigned *scratch, cudaStream_t s) {
    noalloc_step_kernel<R><<<grid, dim3(kTileZ, kNoAllocTY), 0, s>>>(a, scratch + 64);
    return counted(cudaGetLastError(), s);
}

cudaError_t launch_noalloc_r(int r, const StepArgs &a, dim3 grid, unsigned *scratch, cudaStream_t s) {
    switch (r) {
        case 1: return launch_noalloc<1>(a, grid, scratch, s);
        case 2: return launch_noalloc<2>(a, grid, scratch, s);
        case 3: return launch_noalloc<3>(a, grid, scratch, s);
        case 4: return launch_noalloc<4>(a, grid, scratch, s);
        case 5: return launch_noalloc<5>(a, grid, scratch, s);
        case 6: return launch_noalloc<6>(a, grid, scratch, s);
        case 7: return launch_noalloc<7>(a, grid, scratch, s);
        case 8: return launch_noalloc<8>(a, grid, scratch, s);
        default: return cudaErrorInvalidValue;
    }
}

}  // namespace
}  // namespace fdgb

using namespace fdgb;

extern "C" int fd_forward_noalloc(float *d_u, float *d_u_prev, const float *d_m, const float *d_eta,
                                  int Nx, int Ny, int Nz, int space_order, double h, double dt, int ns,
                                  const int *src_xyz, const float *d_wavelet, int ld, long long step0,
                                  int nt, void *stream, float *amax_out) {
    char msg[256];
    auto fail = [&](int code, const char *text) {
        std::snprintf(msg, sizeof msg, "fd_forward_noalloc: %s", text);
        fdgb::set_last_error(msg);
        return code;
    };
    if (!d_u || !d_u_prev || !d_m) return fail(FD_EINVAL, "u, u_prev and m must be device pointers");
    if (Nx < 1 || Ny < 1 || Nz < 1 || Nx > kMaxDim || Ny > kMaxDim || Nz > kMaxDim)
        return fail(FD_EINVAL, "extents must be in [1, 65535]");
    // the library's weight generator (Fornberg's recursion on fixed-size arrays: no heap use)
    double c[kMaxRadiusHost + 1];
    if (space_order > 2 * kNoallocMaxRadius || !fornberg_second_derivative(space_order, c))
        return fail(FD_EINVAL, "space_order must be even in [2, 16]");
    if (!(h > 0) || !std::isfinite(h) || !(dt > 0) || !std::isfinite(dt))
        return fail(FD_EINVAL, "h and dt must be positive and finite");
    if (ns < 0 || ns > kNoallocSources) return fail(FD_EINVAL, "ns must be in [0, 4]");
    if (ns > 0 && (!src_xyz || !d_wavelet || ld < 1)) return fail(FD_EINVAL, "sources need src_xyz, wavelet, ld >= 1");
    if (nt < 0 || step0 < 0) return fail(FD_EINVAL, "nt and step0 must be >= 0");
    const int r = space_order / 2;
    const int tiles_z = (Nz + kTileZ - 1) / kTileZ, tiles_y = (Ny + kNoAllocTY - 1) / kNoAllocTY;
    const long long tiles = (long long)tiles_z * tiles_y;
    if (tiles > kNoAllocMaxCtas)
        return fail(FD_EINVAL, "Ny*Nz too large: one step would need more than 16384 CTAs of scratch");
    // per-device set-up: the address of this device's copy of the scratch array
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kNoAllocMaxDevices)
        return fail(FD_ECUDA, "no usable current device");
    unsigned *scratch = nullptr;
    int sms = 0;
    {
        std::lock_guard<std::mutex> lk(g_noalloc_mu);
        if (!g_noalloc_ptr[dev]) {
            void *p = nullptr;
            cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
            if (e != cudaSuccess) return fail(FD_ECUDA, cudaGetErrorString(e));
            int n_sm = 0;
            e = cudaDeviceGetAttribute(&n_sm, cudaDevAttrMultiProcessorCount, dev);
            if (e != cudaSuccess) return fail(FD_ECUDA, cudaGetErrorString(e));
            g_noalloc_sms[dev] = n_sm > 0 ? n_sm : 1;
            g_noalloc_ptr[dev] = static_cast<unsigned *>(p);
        }
        scratch = g_noalloc_ptr[dev];
        sms = g_noalloc_sms[dev];
    }
    // x-chunks: enough CTAs for four per multiprocessor, within the scratch capacity
    long long chunks = (4LL * sms + tiles - 1) / tiles;
    const long long max_chunks = std::max<long long>(1, std::min<long long>(kNoAllocMaxCtas / tiles, Nx / 16));
    chunks = std::max<long long>(1, std::min(chunks, max_chunks));
    const int x_block = int((Nx + chunks - 1) / chunks);
    const dim3 grid(tiles_z, tiles_y, (Nx + x_block - 1) / x_block);
    const int n_ctas = int(grid.x * grid.y * grid.z);

    StepArgs a{};
    a.f1 = d_m;
    a.f2 = d_eta;
    a.Nx = Nx;
    a.Ny = Ny;
    a.Nz = Nz;
    a.pz = Nz;
    a.plane = (long long)Ny * Nz;
    a.x_block = x_block;
    // no damping field: every point is in the eta-free box, so eta is never read
    if (!d_eta) {
        a.bx1 = Nx;
        a.by1 = Ny;
        a.bz1 = Nz;
    }
    const double scale = dt * dt / (h * h);
    for (int j = 1; j <= r; ++j) a.coef[j] = float(c[j] * scale);
    a.half_dt = float(0.5 * dt);
    a.dt2 = float(dt * dt);
    a.ns = ns;
    for (int s = 0; s < ns; ++s) {
        const int x = src_xyz[3 * s], y = src_xyz[3 * s + 1], z = src_xyz[3 * s + 2];
        if (x < 0 || x >= Nx || y < 0 || y >= Ny || z < 0 || z >= Nz)
            return fail(FD_ERANGE, "source node outside the domain");
        a.sx[s] = x;
        a.sy[s] = y;
        a.sz[s] = z;
    }
    a.wavelet = d_wavelet;
    a.ld = ld;

    cudaStream_t s = static_cast<cudaStream_t>(stream);
    noalloc_clear_kernel<<<1, 32, 0, s>>>(scratch);
    cudaError_t e = counted(cudaGetLastError(), s);
    float *cur = d_u, *prev = d_u_prev;
    for (int i = 0; i < nt && e == cudaSuccess; ++i) {
        a.u = cur;
        a.up = prev;
        a.step = step0 + i;
        e = launch_noalloc_r(r, a, grid, scratch, s);
        if (e == cudaSuccess) {
            noalloc_reduce_kernel<<<1, 256, 0, s>>>(scratch, n_ctas);
            e = counted(cudaGetLastError(), s);
        }
        std::swap(cur, prev);
    }
    if (e != cudaSuccess) return fail(FD_ECUDA, cudaGetErrorString(e));
    if (amax_out) {
        unsigned bits = 0;
        e = cudaMemcpyAsync(&bits, scratch, sizeof bits, cudaMemcpyDeviceToHost, s);
        if (e == cudaSuccess) e = cudaStreamSynchronize(s);
        if (e != cudaSuccess) return fail(FD_ECUDA, cudaGetErrorString(e));
        float v;
        std::memcpy(&v, &bits, sizeof v);
        *amax_out = v;
        if (bits >= 0x7f800000u) return fail(FD_ENONFINITE, "wavefield reached NaN/Inf");
    }
    return FD_OK;
}
