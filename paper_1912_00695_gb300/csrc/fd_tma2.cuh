// Two time steps per launch (temporal blocking along the streaming direction),
// FP32 storage, factored form, stencil radius R <= 2. Included by the radius-1
// and radius-2 translation units after fd_tma.cuh.
//
// Schedule. A CTA of 256 threads owns an extended y-z tile E of 64 (z) x 16 (y)
// points and its interior T (z in [4, 60), y in [R, 16 - R)); neighbouring
// CTAs' extended tiles overlap by their halos. Marching x over the chunk's
// planes extended by R on both sides, at step-1 plane x every thread
//  * computes u^{n+1}(x) at its 4 points of E from u^n (register queue for the
//    x taps, the TMA-fed halo box for y and z, exactly the single-step
//    kernel's per-point arithmetic) and puts it in a shared ring of 2R+1
//    u^{n+1} planes (zero outside the domain: the Dirichlet halo of u^{n+1});
//    points of T inside [xb, xe) are also stored to global memory (u^{n+1});
//  * after a CTA barrier, computes u^{n+2}(x - R) at its points of T from the
//    u^{n+1} ring (x, y and z taps), u^n(x - R) (the oldest queue entry), and
//    w, g of plane x - R (a register queue of R+1 planes), and stores it.
// Per pair of steps HBM sees u^n, u^{n-1}, w (g in the layer) read and
// u^{n+1}, u^{n+2} written: 20 B per point (plus g in the layer) instead of 32
// for two single steps (halo and overlap re-reads come from L2). The extended tile costs
// 64x16 / (56 x (16-2R)) more first-step work. Outputs go to two other
// buffers: u^{n+1} cannot overwrite u^{n-1}, which overlapping CTAs still read.
// Sources of both steps are fused; receivers and the other storages are not
// supported here.
#pragma once

#include "fd_tma.cuh"

namespace fdgb {

template <int R>
struct Tb2Shape {
    static_assert(R >= 1 && R <= 2, "two-step kernel: radius 1 or 2");
    static constexpr int EZ = 64, EY = 16;   // extended tile (z points, y rows)
    static constexpr int HZ = 4;             // z halo of E around T, and of u^n around E (>= R, 16 B)
    static constexpr int TZ = EZ - 2 * HZ;   // 56 output points along z
    static constexpr int TY = EY - 2 * R;    // output rows along y
    static constexpr int SW = EZ + 2 * HZ;   // u^n box width
    static constexpr int SH = EY + 2 * R;    // u^n box height
    static constexpr int HALO_RAW = SW * SH * 4;
    static constexpr int PT_RAW = EZ * EY * 4;
    static constexpr int HALO = (HALO_RAW + 127) / 128 * 128;
    static constexpr int OFF_FRONT = HALO, OFF_UP = HALO + PT_RAW, OFF_F1 = HALO + 2 * PT_RAW,
                         OFF_F2 = HALO + 3 * PT_RAW;
    static constexpr int STAGE_BYTES = HALO + 4 * PT_RAW;
    static constexpr int STAGES = 3;
    static constexpr int NU1 = 2 * R + 1;  // u^{n+1} planes the second step reads
    static constexpr int U1_OFF = STAGES * STAGE_BYTES;
    static constexpr int BAR_OFF = U1_OFF + NU1 * PT_RAW;
    static constexpr int SMEM_BYTES = BAR_OFF + 64 + 128;
    static constexpr int THREADS = 256;
    static constexpr int U = R + 1;  // x unroll: the w/g delay queue indexes statically
};

// Factored FP32 update of 4 points (the single-step kernel's association order):
// L = sum_j c_j ((xm+xp + ym+yp) + z pair - 6 u_c); u+ = w L + (2u - u-) - 2 g (u - u-).
// XT(j, m, p) gives the x taps (m = minus side) as float4; YP(j) the y rows' window
// base (y - j and y + j rows at offsets -j*SW, +j*SW of `rowp`).
template <int R, int RZ, int SWROW, typename XT>
__device__ __forceinline__ float4 tb2_update(const float *rowp, const float *win, XT xtap, float4 uc, float4 cum,
                                             float4 cf1, float4 cf2, const float2 *cz2) {
    float2 lapA = f2(0.f, 0.f), lapB = f2(0.f, 0.f);
    const float2 nsixA = mul2(f2(-6.f, -6.f), lo2(uc)), nsixB = mul2(f2(-6.f, -6.f), hi2(uc));
#pragma unroll
    for (int j = 1; j <= R; ++j) {
        const float4 ym = *reinterpret_cast<const float4 *>(rowp + RZ - j * SWROW);
        const float4 yp = *reinterpret_cast<const float4 *>(rowp + RZ + j * SWROW);
        const float4 xm = xtap(j, true), xp = xtap(j, false);
        const float2 sA = add2(add2(add2(lo2(xm), lo2(xp)), add2(lo2(ym), lo2(yp))), ztap_pair<RZ>(win, j));
        const float2 sB = add2(add2(add2(hi2(xm), hi2(xp)), add2(hi2(ym), hi2(yp))), ztap_pair<RZ + 2>(win, j));
        lapA = fma2(cz2[j], add2(sA, nsixA), lapA);
        lapB = fma2(cz2[j], add2(sB, nsixB), lapB);
    }
    const float2 ucA = lo2(uc), ucB = hi2(uc), umA = lo2(cum), umB = hi2(cum);
    const float2 m2gA = mul2(f2(-2.f, -2.f), lo2(cf2)), m2gB = mul2(f2(-2.f, -2.f), hi2(cf2));
    const float2 dA = fma2(f2(-1.f, -1.f), umA, ucA), dB = fma2(f2(-1.f, -1.f), umB, ucB);
    float2 vA = fma2(lo2(cf1), lapA, add2(ucA, dA));
    float2 vB = fma2(hi2(cf1), lapB, add2(ucB, dB));
    vA = fma2(m2gA, dA, vA);
    vB = fma2(m2gB, dB, vB);
    return make_float4(vA.x, vA.y, vB.x, vB.y);
}

__device__ __forceinline__ float tb2_source(const StepArgs &a, int s, long long step) {
    return (step >= 0 && step < a.ld) ? __ldg(a.wavelet + (long long)s * a.ld + step) : 0.0f;
}

// u^{n+1} into out1 and u^{n+2} into out2 from u^n = a.u, u^{n-1} = a.up (read
// through `maps`), global step n = a.step. CTA (bz, by, bx): T origin
// (bz*56, by*(16-2R)), planes [bx x_block, (bx+1) x_block).
template <int R>
__global__ void __launch_bounds__(256, 2) fd_tma2_kernel(const __grid_constant__ TmaMaps maps, const StepArgs a,
                                                          float *out1, float *out2, int check) {
    using G = Tb2Shape<R>;
    constexpr int S = G::STAGES, U = G::U, Q = 2 * R + U, NWIN = 4 + 2 * G::HZ, EZ = G::EZ, SW = G::SW;
    extern __shared__ __align__(128) unsigned char smem_dyn[];
    // aligned by pointer arithmetic on the shared array (keeps its address space)
    unsigned char *ring = smem_dyn + ((128u - (smem_addr(smem_dyn) & 127u)) & 127u);
    float *u1ring = reinterpret_cast<float *>(ring + G::U1_OFF);
    uint64_t *bars = reinterpret_cast<uint64_t *>(ring + G::BAR_OFF);

    const int tid = threadIdx.x;
    const int lz = tid & 15, ty = tid >> 4;
    const int zt0 = blockIdx.x * G::TZ, yt0 = blockIdx.y * G::TY;
    const int ze0 = zt0 - G::HZ, ye0 = yt0 - R;  // E origin
    const int z4 = ze0 + 4 * lz, y = ye0 + ty;
    const bool dom = y >= 0 && y < a.Ny && z4 >= 0 && z4 < a.Nz;
    const bool inT = lz >= 1 && lz <= 14 && ty >= R && ty < G::EY - R;
    const int xb = blockIdx.z * a.x_block, xe = min(xb + a.x_block, a.Nx);
    const int xs = xb - R, xend = xe + R;  // first-step planes
    const long long P = a.plane;
    const long long col = (long long)y * a.pz + z4;
    const float *u = static_cast<const float *>(a.u) + col;
    float *o1 = out1 + col, *o2 = out2 + col;

    if (tid == 0) {
        for (int s = 0; s < S; ++s) mbar_init(smem_addr(&bars[s]), 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    }
    __syncthreads();
    // the extended tile lies where the damping field vanishes (in y and z)
    const bool tile_yz_box = ye0 >= a.by0 && ye0 + G::EY <= a.by1 && ze0 >= a.bz0 && ze0 + EZ <= a.bz1;
    auto g_free = [&](int x) { return tile_yz_box && x >= a.bx0 && x < a.bx1; };
    auto issue = [&](int x, int stage) {
        const uint32_t bar = smem_addr(&bars[stage]);
        unsigned char *st = ring + stage * G::STAGE_BYTES;
        const bool need_g = !g_free(x);
        mbar_expect_tx(bar, uint32_t(G::HALO_RAW + (need_g ? 4 : 3) * G::PT_RAW));
        tma_load_3d(smem_addr(st), &maps.u_halo, bar, ze0 - G::HZ, ye0 - R, x);
        tma_load_3d(smem_addr(st + G::OFF_FRONT), &maps.u_pt, bar, ze0, ye0, x + R);
        tma_load_3d(smem_addr(st + G::OFF_UP), &maps.up_pt, bar, ze0, ye0, x);
        tma_load_3d(smem_addr(st + G::OFF_F1), &maps.f1_pt, bar, ze0, ye0, x);
        if (need_g) tma_load_3d(smem_addr(st + G::OFF_F2), &maps.f2_pt, bar, ze0, ye0, x);
    };
    const int n_planes = xend - xs;
    if (tid == 0)
        for (int s = 0; s < S - 1 && s < n_planes; ++s) issue(xs + s, s);

    // sources at this thread's 4 points of E: bit s set, sub-index in src_p
    unsigned src_mask = 0;
    int src_p[kFusedSources];
#pragma unroll
    for (int s = 0; s < kFusedSources; ++s) {
        src_p[s] = 0;
        if (dom && s < a.ns && a.sy[s] == y && a.sz[s] >= z4 && a.sz[s] < z4 + 4) {
            src_mask |= 1u << s;
            src_p[s] = a.sz[s] - z4;
        }
    }

    const float4 zero4 = make_float4(0.f, 0.f, 0.f, 0.f);
    auto load_u = [&](int x) -> float4 {
        return (dom && x >= 0 && x < a.Nx) ? __ldg(reinterpret_cast<const float4 *>(u + x * P)) : zero4;
    };
    float4 q[Q];  // u^n at planes xo - R .. xo + R + U - 1 (xo: first plane of the unrolled group)
#pragma unroll
    for (int k = 0; k < 2 * R; ++k) q[k] = load_u(xs - R + k);
    float4 wq[U], gq[U];  // w, g of the last R+1 planes (slot = plane offset within the group)
#pragma unroll
    for (int k = 0; k < U; ++k) wq[k] = gq[k] = zero4;
    float2 cz2[R + 1];
#pragma unroll
    for (int j = 1; j <= R; ++j) cz2[j] = f2(a.coef[j], a.coef[j]);
    const int pt_off = ty * EZ + 4 * lz;  // this thread's 4 points in an E plane
    unsigned amax_bits = 0;
    bool failed = false;
    int issued = min(S - 1, n_planes), it_failed = 0;
    int stage = 0;
    uint32_t phase = 0;

    for (int xo = xs; xo < xend; xo += U) {
#pragma unroll
        for (int i = 0; i < U; ++i) {
            const int x = xo + i;
            if (x >= xend) break;
            const int it = x - xs;
            const bool ok = mbar_wait_bounded(smem_addr(&bars[stage]), phase);
            if (__syncthreads_or(!ok)) {
                failed = true;
                it_failed = it;
                break;
            }
            if (tid == 0 && x + S - 1 < xend) {
                asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
                issue(x + S - 1, stage == 0 ? S - 1 : stage - 1);
                ++issued;
            }
            const unsigned char *st = ring + stage * G::STAGE_BYTES;
            q[2 * R + i] = *reinterpret_cast<const float4 *>(reinterpret_cast<const float *>(st + G::OFF_FRONT) + pt_off);
            // ---- step 1: u^{n+1}(x) at this thread's points of E
            float4 u1 = zero4;
            const float4 cf1 = *reinterpret_cast<const float4 *>(reinterpret_cast<const float *>(st + G::OFF_F1) + pt_off);
            const float4 cf2 = g_free(x) ? zero4
                                         : *reinterpret_cast<const float4 *>(
                                               reinterpret_cast<const float *>(st + G::OFF_F2) + pt_off);
            wq[i] = cf1;
            gq[i] = cf2;
            if (dom && x >= 0 && x < a.Nx) {
                const float4 cum = *reinterpret_cast<const float4 *>(reinterpret_cast<const float *>(st + G::OFF_UP) + pt_off);
                const float *rowp = reinterpret_cast<const float *>(st) + (ty + R) * SW + 4 * lz;
                float win[NWIN];
#pragma unroll
                for (int m = 0; m < NWIN / 4; ++m) {
                    const float4 v = *reinterpret_cast<const float4 *>(rowp + 4 * m);
                    win[4 * m] = v.x;
                    win[4 * m + 1] = v.y;
                    win[4 * m + 2] = v.z;
                    win[4 * m + 3] = v.w;
                }
                u1 = tb2_update<R, G::HZ, SW>(rowp, win, [&](int j, bool minus) { return minus ? q[R + i - j] : q[R + i + j]; },
                                             q[R + i], cum, cf1, cf2, cz2);
                if (src_mask) {
#pragma unroll
                    for (int s = 0; s < kFusedSources; ++s) {
                        if (((src_mask >> s) & 1u) && a.sx[s] == x) {
                            const float qv = tb2_source(a, s, a.step);
                            const int p = src_p[s];
                            if (p == 0) u1.x = fmaf(cf1.x, qv, u1.x);
                            if (p == 1) u1.y = fmaf(cf1.y, qv, u1.y);
                            if (p == 2) u1.z = fmaf(cf1.z, qv, u1.z);
                            if (p == 3) u1.w = fmaf(cf1.w, qv, u1.w);
                        }
                    }
                }
                if (z4 + 3 >= a.Nz) {  // beyond the row's end: zero (the Dirichlet halo and the pitch padding)
                    if (z4 + 1 >= a.Nz) u1.y = 0.f;
                    if (z4 + 2 >= a.Nz) u1.z = 0.f;
                    if (z4 + 3 >= a.Nz) u1.w = 0.f;
                }
                if (inT && x >= xb && x < xe) *reinterpret_cast<float4 *>(o1 + x * P) = u1;
            }
            const int slot1 = it % G::NU1;
            *reinterpret_cast<float4 *>(u1ring + slot1 * (EZ * G::EY) + pt_off) = u1;
            __syncthreads();  // the ring's plane x is complete
            // ---- step 2: u^{n+2}(x - R) at this thread's points of T
            const int x2 = x - R;
            if (inT && dom && x2 >= xb && x2 < xe) {
                const int c0 = (it - R) % G::NU1;  // slot of plane x - R
                const float *plane_c = u1ring + c0 * (EZ * G::EY);
                const float4 uc = *reinterpret_cast<const float4 *>(plane_c + pt_off);
                const float *rowp = plane_c + ty * EZ + 4 * lz - G::HZ;  // z window from 4 points before
                float win[NWIN];
#pragma unroll
                for (int m = 0; m < NWIN / 4; ++m) {
                    const float4 v = *reinterpret_cast<const float4 *>(rowp + 4 * m);
                    win[4 * m] = v.x;
                    win[4 * m + 1] = v.y;
                    win[4 * m + 2] = v.z;
                    win[4 * m + 3] = v.w;
                }
                auto xtap = [&](int j, bool minus) {
                    const int sl = (it - R + (minus ? -j : j) + G::NU1) % G::NU1;
                    return *reinterpret_cast<const float4 *>(u1ring + sl * (EZ * G::EY) + pt_off);
                };
                const float4 w2 = wq[(i + 1) % U], g2 = gq[(i + 1) % U];  // plane x - R
                float4 u2 = tb2_update<R, G::HZ, EZ>(rowp, win, xtap, uc, q[i], w2, g2, cz2);
                if (src_mask) {
#pragma unroll
                    for (int s = 0; s < kFusedSources; ++s) {
                        if (((src_mask >> s) & 1u) && a.sx[s] == x2) {
                            const float qv = tb2_source(a, s, a.step + 1);
                            const int p = src_p[s];
                            if (p == 0) u2.x = fmaf(w2.x, qv, u2.x);
                            if (p == 1) u2.y = fmaf(w2.y, qv, u2.y);
                            if (p == 2) u2.z = fmaf(w2.z, qv, u2.z);
                            if (p == 3) u2.w = fmaf(w2.w, qv, u2.w);
                        }
                    }
                }
                if (z4 + 3 >= a.Nz) {
                    if (z4 + 1 >= a.Nz) u2.y = 0.f;
                    if (z4 + 2 >= a.Nz) u2.z = 0.f;
                    if (z4 + 3 >= a.Nz) u2.w = 0.f;
                }
                amax_bits = max(amax_bits, max(max(__float_as_uint(fabsf(u2.x)), __float_as_uint(fabsf(u2.y))),
                                               max(__float_as_uint(fabsf(u2.z)), __float_as_uint(fabsf(u2.w)))));
                *reinterpret_cast<float4 *>(o2 + x2 * P) = u2;
            }
            if (++stage == S) {
                stage = 0;
                phase ^= 1u;
            }
        }
        if (failed) break;
#pragma unroll
        for (int k = 0; k < 2 * R; ++k) q[k] = q[k + U];
    }
    if (failed) {
        if (tid == 0) {
            if (a.status) atomicOr(a.status, kStatusTimeout);
            for (int it = it_failed; it < issued; ++it) mbar_wait_bounded(smem_addr(&bars[it % S]), uint32_t(it / S) & 1u);
        }
        return;
    }
    if (check) reduce_amax(a, amax_bits, false);
}

template <int R>
cudaError_t tma2_launch(const TmaMaps &maps, const StepArgs &a, float *out1, float *out2, bool check,
                        cudaStream_t s) {
    using G = Tb2Shape<R>;
    auto kernel = fd_tma2_kernel<R>;
    static bool attr_set = false;
    if (!attr_set) {
        cudaError_t e = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, G::SMEM_BYTES);
        if (e != cudaSuccess) return e;
        attr_set = true;
    }
    const dim3 grid((a.Nz + G::TZ - 1) / G::TZ, (a.Ny + G::TY - 1) / G::TY, (a.Nx + a.x_block - 1) / a.x_block);
    kernel<<<grid, G::THREADS, G::SMEM_BYTES, s>>>(maps, a, out1, out2, check ? 1 : 0);
    return cudaGetLastError();
}

}  // namespace fdgb

#define FDGB_INSTANTIATE_TMA2_RADIUS(R)                                                           \
    namespace fdgb {                                                                              \
    cudaError_t tma2_step_radius_##R(const TmaMaps &map, const StepArgs &a, float *out1, float *out2, \
                                     bool check, cudaStream_t s) {                                \
        return tma2_launch<R>(map, a, out1, out2, check, s);                                      \
    }                                                                                             \
    void tma2_geometry_radius_##R(int *tz, int *ty, int *box_w, int *box_h, int *ez, int *ey) {   \
        *tz = Tb2Shape<R>::TZ;                                                                    \
        *ty = Tb2Shape<R>::TY;                                                                    \
        *box_w = Tb2Shape<R>::SW;                                                                 \
        *box_h = Tb2Shape<R>::SH;                                                                 \
        *ez = Tb2Shape<R>::EZ;                                                                    \
        *ey = Tb2Shape<R>::EY;                                                                    \
    }                                                                                             \
    }
