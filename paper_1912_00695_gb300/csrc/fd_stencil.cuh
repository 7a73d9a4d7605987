// Step kernels of the damped acoustic leapfrog (Eq. 1 with the damping term of
// Listing 2), templated on the stencil radius R = k/2, the symbolic form and
// the wavefield storage type. Included by one translation unit per radius.
//
// One launch advances one shot from u^n (args.u) and u^{n-1} (args.up) to
// u^{n+1}, written in place over u^{n-1}: each point reads its own u^{n-1}
// before any thread writes it, and reads of u^n come only from the other
// buffer, so the in-place update is race-free by construction.
#pragma once

#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include "fd_internal.h"

namespace fdgb {

// ---- storage conversions ---------------------------------------------------
template <typename T> struct Io;
template <> struct Io<float> {
    static __device__ __forceinline__ float ldg(const float *p) { return __ldg(p); }
    static __device__ __forceinline__ float ld(const float *p) { return *p; }
    static __device__ __forceinline__ float to_f(float v) { return v; }
    static __device__ __forceinline__ float from_f(float v) { return v; }
    static constexpr bool kScaled = false;
    static constexpr float kMaxStored = 3.0e38f;
};
template <> struct Io<__nv_bfloat16> {
    static __device__ __forceinline__ float ldg(const __nv_bfloat16 *p) {
        return __bfloat162float(__ldg(p));
    }
    static __device__ __forceinline__ float ld(const __nv_bfloat16 *p) { return __bfloat162float(*p); }
    static __device__ __forceinline__ float to_f(__nv_bfloat16 v) { return __bfloat162float(v); }
    static __device__ __forceinline__ __nv_bfloat16 from_f(float v) { return __float2bfloat16_rn(v); }
    static constexpr bool kScaled = true;
    static constexpr float kMaxStored = 3.0e38f;
};
template <> struct Io<__half> {
    static __device__ __forceinline__ float ldg(const __half *p) { return __half2float(__ldg(p)); }
    static __device__ __forceinline__ float ld(const __half *p) { return __half2float(*p); }
    static __device__ __forceinline__ float to_f(__half v) { return __half2float(v); }
    static __device__ __forceinline__ __half from_f(float v) { return __float2half_rn(v); }
    static constexpr bool kScaled = true;
    static constexpr float kMaxStored = 65504.0f;
};

__device__ __forceinline__ int level_slot(long long n) { return int(((n % 3) + 3) % 3); }

// Power-of-two scale mapping `bound` (the largest value expected in the next
// level) to about 2^12, leaving 16x headroom below the FP16 maximum.
__device__ __forceinline__ float pow2_scale(float bound) {
    bound = fmaxf(bound * (1.0f / 4096.0f), 1e-30f);
    int e;
    frexpf(bound, &e);
    return ldexpf(1.0f, e);
}

// Scales of the next levels of a 16-bit shot from max|u^n|, max|d^n| and the
// source bound: d^{n+1} = w L u^n + (1 - 2g) d^n + w q with w L bounded by 4 in
// magnitude below the stability limit, and u^{n+1} = u^n + d^{n+1}.
__device__ __forceinline__ float next_u_scale(float amax_u, float amax_d, float src) {
    return pow2_scale(5.0f * amax_u + amax_d + src);
}
__device__ __forceinline__ float next_d_scale(float amax_u, float amax_d, float src) {
    return pow2_scale(4.0f * amax_u + amax_d + src);
}

// s_u, s_d: scales of the stored u^n and d^n (16-bit) — s_up of u^{n-1} is 1
// for FP32, the only storage of the two-level kernels; inv_s_out, inv_s_d_out:
// reciprocal scales of u^{n+1}, d^{n+1}.
struct ScaleState {
    float s_u, s_up, inv_s_out, s_d, inv_s_d_out, s_out, s_d_out;
};

template <typename T>
__device__ __forceinline__ ScaleState read_scales(const StepArgs &a) {
    ScaleState st{1.0f, 1.0f, 1.0f, 1.0f, 1.0f, 1.0f, 1.0f};
    if constexpr (Io<T>::kScaled) {
        const LevelScales *ls = a.scales;
        const int n = level_slot(a.step);
        st.s_u = ls->scale[n];
        st.s_d = ls->dscale[n];
        const float au = __uint_as_float(ls->amax_bits[n]), ad = __uint_as_float(ls->damax_bits[n]);
        st.s_out = next_u_scale(au, ad, a.src_bound);
        st.s_d_out = next_d_scale(au, ad, a.src_bound);
        st.inv_s_out = 1.0f / st.s_out;  // powers of two: exact
        st.inv_s_d_out = 1.0f / st.s_d_out;
    }
    return st;
}

// One CTA of every launch publishes the scales of u^{n+1}, d^{n+1} and clears
// the max accumulators that the next launch (writing level n+2) will use.
template <typename T>
__device__ __forceinline__ void publish_scales(const StepArgs &a, bool leader) {
    if constexpr (Io<T>::kScaled) {
        if (leader) {
            LevelScales *ls = a.scales;
            const int n = level_slot(a.step), n1 = level_slot(a.step + 1), n2 = level_slot(a.step + 2);
            const float au = __uint_as_float(ls->amax_bits[n]), ad = __uint_as_float(ls->damax_bits[n]);
            ls->scale[n1] = next_u_scale(au, ad, a.src_bound);
            ls->dscale[n1] = next_d_scale(au, ad, a.src_bound);
            ls->amax_bits[n2] = 0u;
            ls->damax_bits[n2] = 0u;
        }
    }
}

// Warp-level max of |u^{n+1}| (and |d^{n+1}| for 16-bit storage) as float bits
// (so NaN > Inf > finite), folded into the level's accumulators and the sticky
// non-finite status bit.
__device__ __forceinline__ void reduce_amax(const StepArgs &a, unsigned bits, bool overflow,
                                            unsigned dbits = 0u) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        bits = max(bits, __shfl_xor_sync(0xffffffffu, bits, o));
        dbits = max(dbits, __shfl_xor_sync(0xffffffffu, dbits, o));
    }
    const unsigned any_over = __any_sync(0xffffffffu, overflow);
    if ((threadIdx.x & 31) == 0) {
        if (a.scales) {
            atomicMax(&a.scales->amax_bits[level_slot(a.step + 1)], bits);
            atomicMax(&a.scales->damax_bits[level_slot(a.step + 1)], dbits);
        }
        if (a.status && (bits >= 0x7f800000u || dbits >= 0x7f800000u || any_over))
            atomicOr(a.status, kStatusNonFinite);
    }
}

// The expanded form's 1/r0, r0 = m + dt/2 eta: the hardware's approximate
// reciprocal (rcp.approx, within 1 ulp; r0 is a normal number), taken once per
// point and step and multiplied into each tap's coefficient. Every kernel of the
// expanded form uses it.
__device__ __forceinline__ float expanded_inv(float r0) {
    float y;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(r0));
    return y;
}

// A point source beyond the fused ones, added to the FP32 level u^{n+1} at
// pitched offset p after the step (its weight: factored w; expanded
// dt^2 / (m + dt/2 eta)); one fused multiply-add. Shared by the per-step
// extra-source kernel and the flow schedule, so both give the same bits.
__device__ __forceinline__ float extra_source_weight(const StepArgs &a, long long p, bool expanded) {
    return expanded ? a.dt2 * expanded_inv(fmaf(a.half_dt, a.f2[p], a.f1[p])) : a.f1[p];
}
__device__ __forceinline__ void add_extra_source_f32(float *level, long long p, float w, float q) {
    level[p] = __fmaf_rn(w, q, level[p]);
}

__device__ __forceinline__ float source_value(const StepArgs &a, int s) {
    return (a.step >= 0 && a.step < a.ld) ? __ldg(a.wavelet + (long long)s * a.ld + a.step) : 0.0f;
}

// The point update shared by both kernels. The Laplacian arrives computed from
// the raw stored values (unscaled) and with the centre folded into every tap:
// since c_0 = -2 sum_j c_j, sum_j c_j (S_j - 6 u_c) equals 3 c_0 u_c + sum_j c_j
// S_j (S_j = the six taps at distance j) but is exactly zero for a locally
// constant field in FP32. A separately rounded centre weight would leave an
// O(ulp) residual that the time loop accumulates as a drift.
// FACTORED: sum_j (c_j/h^2) (S_j - 6 u_c); EXPANDED: every tap (u_tap - u_c)
// times its own per-point coefficient (dt^2 c_j / h^2) / r0.
template <int FORM>
struct Update;

// Factored: u+ = w L u + 2u - u- - 2 g (u - u-), w = dt^2/(m + dt/2 eta),
// g = (dt/2 eta)/(m + dt/2 eta); source weight w.
template <> struct Update<kFactored> {
    static __device__ __forceinline__ float apply(float lap, float uc, float um, float f1, float f2,
                                                  float, const StepArgs &, float &src_w) {
        src_w = f1;
        float v = fmaf(f1, lap, 2.0f * uc - um);
        return fmaf(-2.0f * f2, uc - um, v);
    }
};
// Expanded: u+ = sum_taps (dt^2 c/h^2 / r0) u_tap + (2m/r0) u + ((dt/2 eta - m)/r0) u-,
// r0 = m + dt/2 eta; the tap sum arrives already divided by r0 (times 1/r0).
// The two level coefficients are formed from a = m/r0 by a correctly rounded
// division, so that in the undamped interior they are exactly 2 and -1: a
// reciprocal-multiply would bias them by an ulp in the same direction at every
// step and the bias would accumulate over the time loop. Source weight dt^2/r0.
template <> struct Update<kExpanded> {
    static __device__ __forceinline__ float apply(float taps, float uc, float um, float m, float e,
                                                  float inv, const StepArgs &a, float &src_w) {
        src_w = a.dt2 * inv;
        const float am = __fdiv_rn(m, fmaf(a.half_dt, e, m));
        float v = fmaf(2.0f * am, uc, taps);
        return fmaf(1.0f - 2.0f * am, um, v);
    }
};

// ---- naive kernel: one thread per point, every tap from global memory ------
template <int R, int FORM, typename T>
__global__ void __launch_bounds__(256) fd_naive_kernel(const StepArgs a, int check) {
    static_assert(!Io<T>::kScaled, "16-bit storage runs on the TMA kernel (increment form)");
    const int z = blockIdx.x * 32 + threadIdx.x;
    const int y = blockIdx.y * 8 + threadIdx.y;
    const int x = blockIdx.z;
    const bool own = (z < a.Nz) && (y < a.Ny);
    const T *__restrict__ u = static_cast<const T *>(a.u);
    T *up = static_cast<T *>(a.up);
    const ScaleState sc = read_scales<T>(a);
    publish_scales<T>(a, blockIdx.x == 0 && blockIdx.y == 0 && blockIdx.z == 0 && threadIdx.x == 0 &&
                             threadIdx.y == 0);
    unsigned amax_bits = 0;
    bool over = false;
    if (own) {
        const long long p = (long long)x * a.plane + (long long)y * a.pz + z;
        auto at = [&](int xx, int yy, int zz) -> float {
            if (xx < 0 || xx >= a.Nx || yy < 0 || yy >= a.Ny || zz < 0 || zz >= a.Nz) return 0.0f;
            return Io<T>::ldg(u + (long long)xx * a.plane + (long long)yy * a.pz + zz);
        };
        const float uc = at(x, y, z);
        const float um = Io<T>::ld(up + p) * sc.s_up;
        const bool in_box = x >= a.bx0 && x < a.bx1 && y >= a.by0 && y < a.by1 && z >= a.bz0 &&
                            z < a.bz1;
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
            v = Update<kFactored>::apply(lap * sc.s_u, uc * sc.s_u, um, f1, f2, 0.0f, a, src_w);
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
            v = Update<kExpanded>::apply(taps * sc.s_u, uc * sc.s_u, um, f1, f2, inv, a, src_w);
        }
        for (int s = 0; s < a.ns && s < kFusedSources; ++s)
            if (a.sx[s] == x && a.sy[s] == y && a.sz[s] == z) v = fmaf(src_w, source_value(a, s), v);
        const float stored = v * sc.inv_s_out;
        if constexpr (Io<T>::kScaled) over = fabsf(stored) > Io<T>::kMaxStored;
        up[p] = Io<T>::from_f(stored);
        amax_bits = __float_as_uint(fabsf(v));
    }
    if (check) reduce_amax(a, amax_bits, over);
}

// ---- streaming kernel --------------------------------------------------------
// CTA = 32 (z) x TY (y) threads, one output column (y, z) per thread, marching
// x over [x0, x0 + x_block). Each thread keeps u^n at x-R..x+R of its column in
// a register queue (the x taps); the current x-plane of u^n, with a halo of R
// cells in y and z, sits in a double-buffered shared tile (the y and z taps).
// Halo values and the next plane's point data are prefetched into registers
// one plane ahead, so each plane costs one barrier.
template <int R, int FORM, int TY, typename T>
__global__ void __launch_bounds__(32 * TY) fd_stream_kernel(const StepArgs a, int check) {
    static_assert(!Io<T>::kScaled, "16-bit storage runs on the TMA kernel (increment form)");
    constexpr int TZ = kTileZ;
    constexpr int SW = TZ + 2 * R;
    constexpr int SH = TY + 2 * R;
    constexpr int NYH = (R + TY - 1) / TY;
    __shared__ T tile[2][SH][SW];

    const int tz = threadIdx.x, ty = threadIdx.y;
    const int z0 = blockIdx.x * TZ, y0 = blockIdx.y * TY;
    const int z = z0 + tz, y = y0 + ty;
    const int xb = blockIdx.z * a.x_block;
    const int xe = min(xb + a.x_block, a.Nx);
    const bool own = (y < a.Ny) && (z < a.Nz);
    const T *__restrict__ u = static_cast<const T *>(a.u);
    T *up = static_cast<T *>(a.up);
    const long long P = a.plane;
    const long long col = (long long)y * a.pz + z;
    const bool yz_box = y >= a.by0 && y < a.by1 && z >= a.bz0 && z < a.bz1;

    const ScaleState sc = read_scales<T>(a);
    publish_scales<T>(a, blockIdx.x == 0 && blockIdx.y == 0 && blockIdx.z == 0 && tz == 0 && ty == 0);

    // sources in this thread's column
    unsigned src_mask = 0;
    if (own)
        for (int s = 0; s < a.ns && s < kFusedSources; ++s)
            if (a.sy[s] == y && a.sz[s] == z && a.sx[s] >= xb && a.sx[s] < xe) src_mask |= 1u << s;

    // halo registers for one plane
    T hy_lo[NYH], hy_hi[NYH], hz_lo, hz_hi;
    const T zero = Io<T>::from_f(0.0f);
    auto load_halo = [&](int x) {
        const long long px = (long long)x * P;
#pragma unroll
        for (int k = 0; k < NYH; ++k) {
            const int i = ty + k * TY;
            hy_lo[k] = zero;
            hy_hi[k] = zero;
            if (i < R && z < a.Nz) {
                const int ya = y0 - R + i, yb = y0 + TY + i;
                if (ya >= 0) hy_lo[k] = __ldg(u + px + (long long)ya * a.pz + z);
                if (yb < a.Ny) hy_hi[k] = __ldg(u + px + (long long)yb * a.pz + z);
            }
        }
        hz_lo = zero;
        hz_hi = zero;
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
        return (own && x >= 0 && x < a.Nx) ? Io<T>::ldg(u + (long long)x * P + col) : 0.0f;
    };

    float q[2 * R + 1];
#pragma unroll
    for (int i = 0; i < 2 * R; ++i) q[i] = load_u(xb - R + i);
    float nxt = load_u(xb + R);
    load_halo(xb);
    float pum = 0.0f, pf1 = 0.0f, pf2 = 0.0f;
    auto load_point = [&](int x) {
        if (own) {
            const long long p = (long long)x * P + col;
            pum = Io<T>::ld(up + p);
            pf1 = __ldg(a.f1 + p);
            const bool in_box = yz_box && x >= a.bx0 && x < a.bx1;
            pf2 = in_box ? 0.0f : __ldg(a.f2 + p);
        }
    };
    load_point(xb);

    unsigned amax_bits = 0;
    bool over = false;
    for (int x = xb; x < xe; ++x) {
        const int buf = (x - xb) & 1;
        q[2 * R] = nxt;
        store_halo(buf);
        tile[buf][ty + R][tz + R] = Io<T>::from_f(q[R]);
        __syncthreads();
        const float cum = pum, cf1 = pf1, cf2 = pf2;
        if (x + 1 < xe) {
            load_halo(x + 1);
            nxt = load_u(x + 1 + R);
            load_point(x + 1);
        }
        if (own) {
            const T(*t)[SW] = tile[buf];
            const int cy = ty + R, cz = tz + R;
            const float uc = q[R];
            float v, src_w;
            if constexpr (FORM == kFactored) {
                const float six_uc = 6.0f * uc;
                float lap = 0.0f;
#pragma unroll
                for (int j = 1; j <= R; ++j) {
                    const float s = (q[R - j] + q[R + j]) +
                                    (Io<T>::to_f(t[cy - j][cz]) + Io<T>::to_f(t[cy + j][cz])) +
                                    (Io<T>::to_f(t[cy][cz - j]) + Io<T>::to_f(t[cy][cz + j]));
                    lap = fmaf(a.coef[j], s - six_uc, lap);
                }
                v = Update<kFactored>::apply(lap * sc.s_u, uc * sc.s_u, cum * sc.s_up, cf1, cf2, 0.0f,
                                             a, src_w);
            } else {
                const float inv = expanded_inv(fmaf(a.half_dt, cf2, cf1));
                float taps = 0.0f;
#pragma unroll
                for (int j = 1; j <= R; ++j) {
                    const float cj = a.coef[j] * inv;
                    taps = fmaf(cj, q[R - j] - uc, taps);
                    taps = fmaf(cj, q[R + j] - uc, taps);
                    taps = fmaf(cj, Io<T>::to_f(t[cy - j][cz]) - uc, taps);
                    taps = fmaf(cj, Io<T>::to_f(t[cy + j][cz]) - uc, taps);
                    taps = fmaf(cj, Io<T>::to_f(t[cy][cz - j]) - uc, taps);
                    taps = fmaf(cj, Io<T>::to_f(t[cy][cz + j]) - uc, taps);
                }
                v = Update<kExpanded>::apply(taps * sc.s_u, uc * sc.s_u, cum * sc.s_up, cf1, cf2, inv,
                                             a, src_w);
            }
            if (src_mask) {
#pragma unroll
                for (int s = 0; s < kFusedSources; ++s)
                    if (((src_mask >> s) & 1u) && a.sx[s] == x) v = fmaf(src_w, source_value(a, s), v);
            }
            const float stored = v * sc.inv_s_out;
            if constexpr (Io<T>::kScaled) over |= fabsf(stored) > Io<T>::kMaxStored;
            up[(long long)x * P + col] = Io<T>::from_f(stored);
            amax_bits = max(amax_bits, __float_as_uint(fabsf(v)));
        }
#pragma unroll
        for (int i = 0; i < 2 * R; ++i) q[i] = q[i + 1];
    }
    if (check) reduce_amax(a, amax_bits, over);
}

// ---- dispatch for one radius ---------------------------------------------------
template <int R>
cudaError_t stream_step_r(int form, int storage, int tile_y, const StepArgs &a, bool check,
                          cudaStream_t s) {
    const dim3 grid((a.Nz + kTileZ - 1) / kTileZ, 0, (a.Nx + a.x_block - 1) / a.x_block);
    auto go = [&](auto kernel, int ty) {
        dim3 g(grid.x, (a.Ny + ty - 1) / ty, grid.z);
        kernel<<<g, dim3(kTileZ, ty), 0, s>>>(a, check ? 1 : 0);
        return cudaGetLastError();
    };
#define FDGB_STREAM_CASE(FORM, T)                                                        \
    switch (tile_y) {                                                                    \
        case 4: return go(fd_stream_kernel<R, FORM, 4, T>, 4);                           \
        case 8: return go(fd_stream_kernel<R, FORM, 8, T>, 8);                           \
        case 16: return go(fd_stream_kernel<R, FORM, 16, T>, 16);                        \
        default: return cudaErrorInvalidValue;                                           \
    }
    if (storage != kF32) return cudaErrorInvalidValue;
    if (form == kFactored) {
        FDGB_STREAM_CASE(kFactored, float)
    } else {
        FDGB_STREAM_CASE(kExpanded, float)
    }
#undef FDGB_STREAM_CASE
    return cudaErrorInvalidValue;
}

template <int R>
cudaError_t naive_step_r(int form, int storage, const StepArgs &a, bool check, cudaStream_t s) {
    const dim3 grid((a.Nz + 31) / 32, (a.Ny + 7) / 8, a.Nx);
    const dim3 block(32, 8);
    const int c = check ? 1 : 0;
    if (storage != kF32) return cudaErrorInvalidValue;
    if (form == kFactored) fd_naive_kernel<R, kFactored, float><<<grid, block, 0, s>>>(a, c);
    else fd_naive_kernel<R, kExpanded, float><<<grid, block, 0, s>>>(a, c);
    return cudaGetLastError();
}

}  // namespace fdgb

#define FDGB_INSTANTIATE_RADIUS(R)                                                                \
    namespace fdgb {                                                                              \
    cudaError_t stream_step_radius_##R(int form, int storage, int tile_y, const StepArgs &a,     \
                                       bool check, cudaStream_t s) {                             \
        return stream_step_r<R>(form, storage, tile_y, a, check, s);                              \
    }                                                                                             \
    cudaError_t naive_step_radius_##R(int form, int storage, const StepArgs &a, bool check,       \
                                      cudaStream_t s) {                                           \
        return naive_step_r<R>(form, storage, a, check, s);                                       \
    }                                                                                             \
    }
