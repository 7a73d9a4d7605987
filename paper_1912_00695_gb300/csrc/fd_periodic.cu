// Periodic-boundary step: the test mode in which the computational domain is
// a 3-torus. This is the setting of the scheme's closed-form solutions (a
// discrete plane wave cos(k.x - w t) whose frequency obeys the scheme's
// dispersion relation) and of its conserved discrete energy when eta = 0, so
// tests can check the GPU path against the mathematics directly. The per-point
// arithmetic is the naive kernel's (same expression order, both forms); only
// the tap indices differ: taken modulo the extent instead of reading a zero
// halo. One thread per point, FP32 storage, fused sources (the first four).
#include "fd_launch_count.h"
#include "fd_periodic.h"
#include "fd_stencil.cuh"

namespace fdgb {
namespace {

__device__ __forceinline__ int wrap(int i, int n) {
    i %= n;
    return i < 0 ? i + n : i;
}

template <int R, int FORM>
__global__ void __launch_bounds__(256) fd_periodic_kernel(const StepArgs a, int check) {
    const int z = blockIdx.x * 32 + threadIdx.x;
    const int y = blockIdx.y * 8 + threadIdx.y;
    const int x = blockIdx.z;
    unsigned amax_bits = 0;
    if (z < a.Nz && y < a.Ny) {
        const float *__restrict__ u = static_cast<const float *>(a.u);
        float *up = static_cast<float *>(a.up);
        const long long p = (long long)x * a.plane + (long long)y * a.pz + z;
        auto at = [&](int xx, int yy, int zz) -> float {
            return __ldg(u + (long long)wrap(xx, a.Nx) * a.plane + (long long)wrap(yy, a.Ny) * a.pz +
                         wrap(zz, a.Nz));
        };
        const float uc = __ldg(u + p);
        const float um = up[p];
        const bool in_box = x >= a.bx0 && x < a.bx1 && y >= a.by0 && y < a.by1 && z >= a.bz0 && z < a.bz1;
        const float f1 = __ldg(a.f1 + p);
        const float f2 = in_box ? 0.0f : __ldg(a.f2 + p);
        float v, src_w;
        if constexpr (FORM == kFactored) {
            const float six_uc = 6.0f * uc;
            float lap = 0.0f;
#pragma unroll
            for (int j = 1; j <= R; ++j) {
                const float s = (at(x - j, y, z) + at(x + j, y, z)) + (at(x, y - j, z) + at(x, y + j, z)) +
                                (at(x, y, z - j) + at(x, y, z + j));
                lap = fmaf(a.coef[j], s - six_uc, lap);
            }
            v = Update<kFactored>::apply(lap, uc, um, f1, f2, 0.0f, a, src_w);
        } else {
            const float inv = expanded_inv(fmaf(a.half_dt, f2, f1));
            float taps = 0.0f;
#pragma unroll
            for (int j = 1; j <= R; ++j) {
                const float cj = a.coef[j] * inv;
                taps = fmaf(cj, at(x - j, y, z) - uc, taps);
                taps = fmaf(cj, at(x + j, y, z) - uc, taps);
                taps = fmaf(cj, at(x, y - j, z) - uc, taps);
                taps = fmaf(cj, at(x, y + j, z) - uc, taps);
                taps = fmaf(cj, at(x, y, z - j) - uc, taps);
                taps = fmaf(cj, at(x, y, z + j) - uc, taps);
            }
            v = Update<kExpanded>::apply(taps, uc, um, f1, f2, inv, a, src_w);
        }
        for (int s = 0; s < a.ns && s < kFusedSources; ++s)
            if (a.sx[s] == x && a.sy[s] == y && a.sz[s] == z) v = fmaf(src_w, source_value(a, s), v);
        up[p] = v;
        amax_bits = __float_as_uint(fabsf(v));
    }
    if (check) reduce_amax(a, amax_bits, false);
}

template <int R>
cudaError_t periodic_step_r(int form, const StepArgs &a, bool check, cudaStream_t s) {
    const dim3 grid((a.Nz + 31) / 32, (a.Ny + 7) / 8, a.Nx);
    const dim3 block(32, 8);
    if (form == kFactored) fd_periodic_kernel<R, kFactored><<<grid, block, 0, s>>>(a, check ? 1 : 0);
    else fd_periodic_kernel<R, kExpanded><<<grid, block, 0, s>>>(a, check ? 1 : 0);
    return cudaGetLastError();
}

}  // namespace

cudaError_t launch_periodic_step(int radius, int form, const StepArgs &a, bool check, cudaStream_t s) {
    cudaError_t e = cudaErrorInvalidValue;
    switch (radius) {
        case 1: e = periodic_step_r<1>(form, a, check, s); break;
        case 2: e = periodic_step_r<2>(form, a, check, s); break;
        case 3: e = periodic_step_r<3>(form, a, check, s); break;
        case 4: e = periodic_step_r<4>(form, a, check, s); break;
        case 5: e = periodic_step_r<5>(form, a, check, s); break;
        case 6: e = periodic_step_r<6>(form, a, check, s); break;
        case 7: e = periodic_step_r<7>(form, a, check, s); break;
        case 8: e = periodic_step_r<8>(form, a, check, s); break;
        case 9: e = periodic_step_r<9>(form, a, check, s); break;
        case 10: e = periodic_step_r<10>(form, a, check, s); break;
        case 11: e = periodic_step_r<11>(form, a, check, s); break;
        case 12: e = periodic_step_r<12>(form, a, check, s); break;
        default: return cudaErrorInvalidValue;
    }
    return counted(e, s);
}

}  // namespace fdgb
