// TMA-fed streaming step kernel, templated on the stencil radius R, the
// symbolic form, the tile shape and the wavefield storage type T (float,
// bfloat16, half). Included by the per-radius translation units after
// fd_stencil.cuh.
//
// Schedule. A CTA of W warps owns a tile of TZ = 4*LZ points along z by
// TY = (32/LZ)*W points along y and marches x over [x0, x0 + x_block). Each
// thread owns 4 consecutive z points of one y row:
//  * x taps: a register queue of 4-point vectors (u^n at x-R..x+R of the
//    thread's points); the x loop is unrolled by U planes and the queue shifts
//    by U once per U planes (2R/U vector moves per plane, code size U bodies);
//  * y and z taps: the current x-plane of u^n with an R-cell halo (z halo
//    rounded up so every TMA box starts 16-byte aligned), fetched by one
//    tensor-map bulk copy per plane into a shared ring guarded by mbarriers;
//    out-of-domain boxes are zero-filled by the copy engine, which is exactly
//    the Dirichlet halo;
//  * the queue front u^n(x+R) and the point data u^{n-1}, w (m), g (eta) of
//    plane x arrive in the same ring stage as its halo tile (one bulk tensor
//    copy each, several planes ahead, g skipped where the damping vanishes),
//    so no thread waits on a global load inside the loop; further ahead the
//    same boxes are pulled into L2 by bulk tensor prefetches; the result is
//    one vector store;
//  * the arithmetic runs in FP32 on float2 pairs (FFMA2/FADD2), two points per
//    instruction;
//  * 16-bit storage keeps u^n and the increment d^n = u^n - u^{n-1} (the
//    discrete velocity times dt), each with its own per-level power-of-two
//    scale: d^{n+1} = w L u^n + (1 - 2g) d^n + w q, u^{n+1} = u^n + d^{n+1}.
//    Rounding both leapfrog levels instead would cost the velocity u - u^{-}
//    about ulp/(omega dt) of relative precision per step, which grows without
//    bound over long runs. Values are converted on load and scaled; the
//    Laplacian is linear, so it is computed on the raw values and scaled once.
// The per-point arithmetic (association order included) does not depend on
// the tile shape or x_block.
#pragma once

#include <cuda.h>

#include "fd_stencil.cuh"

namespace fdgb {

// Ring depth: planes whose inputs are in flight or resident in shared memory,
// sized so that four 128-thread CTAs (16 warps) fit an SM's shared memory with
// the 32x16 tile.
template <int R>
struct TmaPipe {
    static constexpr int STAGES = R >= 7 ? 3 : 4;
};
constexpr long long kMbarWaitLimit = 1LL << 22;
constexpr int kPrefetchAhead = 6;  // planes between the L2 prefetch and the register load

__device__ __forceinline__ uint32_t smem_addr(const void *p) {
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void mbar_init(uint32_t bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_expect_tx(uint32_t bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes)
                 : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint32_t bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(bar), "r"(parity)
        : "memory");
    return ok != 0;
}

// Nanoseconds of the GPU's global timer.
__device__ __forceinline__ unsigned long long global_ns() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

constexpr unsigned long long kMbarWaitNs = 1000000000ull;  // a ring wait gives up after 1 s

// Bounded wait: gives up after kMbarWaitNs of the global timer (or kMbarWaitLimit
// polls, whichever comes first), so that a copy that never lands cannot hang the GPU.
__device__ __forceinline__ bool mbar_wait_bounded(uint32_t bar, uint32_t parity) {
    unsigned long long t0 = 0;
    for (long long i = 0; i < kMbarWaitLimit; ++i) {
        if (mbar_try_wait(bar, parity)) return true;
        if (i >= 8) {
            if (i == 8) t0 = global_ns();
            else if (global_ns() - t0 > kMbarWaitNs) return false;
            __nanosleep(64);
        }
    }
    return false;
}

__device__ __forceinline__ void tma_load_3d(uint32_t dst, const CUtensorMap *map, uint32_t bar,
                                            int c0, int c1, int c2) {
    asm volatile(
        "cp.async.bulk.tensor.3d.shared::cluster.global.tile.mbarrier::complete_tx::bytes "
        "[%0], [%1, {%3, %4, %5}], [%2];" ::"r"(dst),
        "l"(reinterpret_cast<uint64_t>(map)), "r"(bar), "r"(c0), "r"(c1), "r"(c2)
        : "memory");
}

__device__ __forceinline__ void tma_load_4d(uint32_t dst, const CUtensorMap *map, uint32_t bar, int c0, int c1, int c2,
                                            int c3) {
    asm volatile(
        "cp.async.bulk.tensor.4d.shared::cluster.global.tile.mbarrier::complete_tx::bytes "
        "[%0], [%1, {%3, %4, %5, %6}], [%2];" ::"r"(dst),
        "l"(reinterpret_cast<uint64_t>(map)), "r"(bar), "r"(c0), "r"(c1), "r"(c2), "r"(c3)
        : "memory");
}

__device__ __forceinline__ void tma_prefetch_3d(const CUtensorMap *map, int c0, int c1, int c2) {
    asm volatile("cp.async.bulk.prefetch.tensor.3d.L2.global.tile [%0, {%1, %2, %3}];" ::"l"(
                     reinterpret_cast<uint64_t>(map)),
                 "r"(c0), "r"(c1), "r"(c2)
                 : "memory");
}

__device__ __forceinline__ float2 f2(float a, float b) { return make_float2(a, b); }
__device__ __forceinline__ float2 lo2(const float4 &v) { return make_float2(v.x, v.y); }
__device__ __forceinline__ float2 hi2(const float4 &v) { return make_float2(v.z, v.w); }
__device__ __forceinline__ float2 add2(float2 a, float2 b) { return __fadd2_rn(a, b); }
__device__ __forceinline__ float2 sub2(float2 a, float2 b) { return __fadd2_rn(a, make_float2(-b.x, -b.y)); }
__device__ __forceinline__ float2 mul2(float2 a, float2 b) { return __fmul2_rn(a, b); }
__device__ __forceinline__ float2 fma2(float2 a, float2 b, float2 c) { return __ffma2_rn(a, b, c); }

// Four consecutive stored values <-> float4 (raw, unscaled).
template <typename T> struct Vec4;
template <> struct Vec4<float> {
    static constexpr CUtensorMapDataType kMapType = CU_TENSOR_MAP_DATA_TYPE_FLOAT32;
    static __device__ __forceinline__ float4 ldg(const float *p) { return __ldg(reinterpret_cast<const float4 *>(p)); }
    // cached in L2 only: data other CTAs of the same launch may have written
    static __device__ __forceinline__ float4 ldcg(const float *p) { return __ldcg(reinterpret_cast<const float4 *>(p)); }
    static __device__ __forceinline__ float4 ld(const float *p) { return *reinterpret_cast<const float4 *>(p); }
    static __device__ __forceinline__ void st(float *p, float4 v) { *reinterpret_cast<float4 *>(p) = v; }
};
template <typename H, typename H2> struct Vec4Half {
    static __device__ __forceinline__ float2 to2(H2 v);
    static __device__ __forceinline__ H2 from2(float2 v);
    static __device__ __forceinline__ float4 cvt(uint2 r) {
        const float2 a = to2(*reinterpret_cast<const H2 *>(&r.x)), b = to2(*reinterpret_cast<const H2 *>(&r.y));
        return make_float4(a.x, a.y, b.x, b.y);
    }
    static __device__ __forceinline__ float4 ldg(const H *p) { return cvt(__ldg(reinterpret_cast<const uint2 *>(p))); }
    // cached in L2 only: data other CTAs of the same launch may have written
    static __device__ __forceinline__ float4 ldcg(const H *p) { return cvt(__ldcg(reinterpret_cast<const uint2 *>(p))); }
    static __device__ __forceinline__ float4 ld(const H *p) { return cvt(*reinterpret_cast<const uint2 *>(p)); }
    static __device__ __forceinline__ void st(H *p, float4 v) {
        uint2 r;
        *reinterpret_cast<H2 *>(&r.x) = from2(make_float2(v.x, v.y));
        *reinterpret_cast<H2 *>(&r.y) = from2(make_float2(v.z, v.w));
        *reinterpret_cast<uint2 *>(p) = r;
    }
};
template <> __device__ __forceinline__ float2 Vec4Half<__nv_bfloat16, __nv_bfloat162>::to2(__nv_bfloat162 v) {
    return __bfloat1622float2(v);
}
template <> __device__ __forceinline__ __nv_bfloat162 Vec4Half<__nv_bfloat16, __nv_bfloat162>::from2(float2 v) {
    return __float22bfloat162_rn(v);
}
template <> __device__ __forceinline__ float2 Vec4Half<__half, __half2>::to2(__half2 v) { return __half22float2(v); }
template <> __device__ __forceinline__ __half2 Vec4Half<__half, __half2>::from2(float2 v) {
    return __float22half2_rn(v);
}
template <> struct Vec4<__nv_bfloat16> : Vec4Half<__nv_bfloat16, __nv_bfloat162> {};
template <> struct Vec4<__half> : Vec4Half<__half, __half2> {};

template <int R, int LZ, int W, typename T, int EXTRA_F = 0, int YB = 1>
struct TmaShape {
    static constexpr int VE = 16 / int(sizeof(T));         // elements per 16 bytes
    static constexpr int RZ = (R + VE - 1) / VE * VE;       // z halo: boxes start 16-byte aligned
    static constexpr int LY = 32 / LZ;
    static constexpr int TZ = 4 * LZ;
    static constexpr int TY = LY * W * YB;  // YB rows per thread
    static constexpr int SW = TZ + 2 * RZ;  // box width (elements)
    static constexpr int SH = TY + 2 * R;   // box height (rows)
    // one ring stage: the halo tile of u^n(x), then the point tiles (TZ x TY, no halo)
    // of the queue front u^n(x+R), of u^{n-1}(x) (16-bit: d^n(x)), w(x) and g(x)
    static constexpr int HALO_RAW = SW * SH * int(sizeof(T));
    static constexpr int PT_T_RAW = TZ * TY * int(sizeof(T));
    static constexpr int PT_F_RAW = TZ * TY * 4;
    static constexpr int HALO = (HALO_RAW + 127) / 128 * 128;
    static constexpr int PT_T = (PT_T_RAW + 127) / 128 * 128;
    static constexpr int PT_F = (PT_F_RAW + 127) / 128 * 128;
    static constexpr int OFF_FRONT = HALO, OFF_UP = HALO + PT_T, OFF_F1 = HALO + 2 * PT_T,
                         OFF_F2 = HALO + 2 * PT_T + PT_F;
    // EXTRA_F more FP32 point tiles (the gradient pass: D^{k-1}, then the gradient)
    static constexpr int OFF_X0 = HALO + 2 * PT_T + 2 * PT_F, OFF_X1 = OFF_X0 + PT_F;
    static constexpr int STAGE_BYTES = HALO + 2 * PT_T + (2 + EXTRA_F) * PT_F;
    // the mbarriers (first 128 bytes), then the stages, plus slack to align to 128 bytes
    // (bulk tensor copies need a 128-byte aligned shared destination)
    static constexpr int SMEM_BYTES = 128 + TmaPipe<R>::STAGES * STAGE_BYTES + 128;
};

// x-loop unroll (planes per queue shift): deeper unrolling saves queue moves but
// grows the loop body; at R >= 5 the body of 2 planes measured fastest.
template <int R, int FORM>
struct TmaUnroll {
    static constexpr int U = FORM == kFactored ? (R >= 5 ? 2 : 4) : 2;
};

// Sum of the two z taps at distance j of the pair of points (p, p+1) whose
// window index is W0 = RZ + p: (win[W0-j] + win[W0+j], win[W0+1-j] + win[W0+1+j]).
// When W0 - j is even both operand pairs are aligned register pairs and one
// paired add does it; otherwise two scalar adds write an aligned result pair
// directly (cheaper than re-pairing misaligned operands).
template <int W0>
__device__ __forceinline__ float2 ztap_pair(const float *win, int j) {
    if (((W0 - j) & 1) == 0)
        return __fadd2_rn(make_float2(win[W0 - j], win[W0 + 1 - j]), make_float2(win[W0 + j], win[W0 + 1 + j]));
    return make_float2(win[W0 - j] + win[W0 + j], win[W0 + 1 - j] + win[W0 + 1 + j]);
}

// (win[W0 + o] - u.x, win[W0 + 1 + o] - u.y) for the pair (p, p+1) at window index W0
// = RZ + p and tap offset o: one paired subtraction when the operands form an
// aligned register pair (W0 + o even), else two scalar ones writing an aligned
// result pair (the same roundings either way).
template <int W0>
__device__ __forceinline__ float2 zdiff_pair(const float *win, int o, float2 u) {
    if (((W0 + o) & 1) == 0) return __fadd2_rn(make_float2(win[W0 + o], win[W0 + 1 + o]), make_float2(-u.x, -u.y));
    return make_float2(win[W0 + o] - u.x, win[W0 + 1 + o] - u.y);
}

// Per-CTA accumulators of the max-|value| reduction, carried across segments.
struct TmaAcc {
    unsigned amax_bits = 0, damax_bits = 0;
    bool over = false;
};

// The ring of stages in dynamic shared memory (128-byte aligned) and its S
// mbarriers; thread 0 initialises the barriers once per CTA.
template <int R>
__device__ __forceinline__ unsigned char *tma_ring_init(unsigned char *smem_raw) {
    constexpr int S = TmaPipe<R>::STAGES;
    // the S mbarriers sit in the first 128 bytes, the ring right after them, so their
    // place does not depend on the stage layout
    // aligned by pointer arithmetic on the shared array itself (not through an
    // integer), so that the compiler keeps its address space and every access to
    // the ring is a shared-memory load with 32-bit addressing
    unsigned char *base = smem_raw + ((128u - (smem_addr(smem_raw) & 127u)) & 127u);
    unsigned char *ring = base + 128;
    if (threadIdx.x == 0) {
        uint64_t *bars = reinterpret_cast<uint64_t *>(base);
        for (int s = 0; s < S; ++s) mbar_init(smem_addr(&bars[s]), 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    }
    __syncthreads();
    return ring;
}

// One segment of a CTA's work: planes [xb, xe) of tile (bz, by) of the y-z plane
// of the shot described by `a` and `maps`. `g` counts the planes the CTA has
// already streamed through its ring (it selects the stage and the mbarrier
// phase, so consecutive segments share one ring without re-initialising it).
// Returns false if a wait gave up (status set, copies in flight drained).
// COHERENT: u^n may have been written earlier in the same launch (the flow
// schedule), so the queue prologue reads it through L2 instead of the
// read-only path. step >= 0 replaces a.step (the flow schedule's steps share
// one argument block).
// YB: y rows per thread (1 or 2). With two adjacent rows a thread loads each
// y-tap row of the halo tile once for both (2R + 2 row loads for 8 points
// instead of 2 (2R + 1)), carries twice the independent accumulation chains
// and meets one CTA barrier per 8 points instead of 4; its x queues take
// twice the registers, so such CTAs run at half the warps per SM. The
// per-point arithmetic and its order are those of one row per thread.
template <int R, int FORM, int LZ, int W, typename T, int MODE = kModeStep, bool COHERENT = false, int YB = 1>
__device__ __forceinline__ bool tma_segment(const TmaMaps *maps, const StepArgs &a, const ScaleState &sc, int bz,
                                            int by, int xb, int xe, unsigned char *ring, int &g, TmaAcc &acc,
                                            const GradMaps *gm = nullptr, long long step = -1) {
    using G = TmaShape<R, LZ, W, T, MODE == kModeAdjointGrad ? 2 : 0, YB>;
    using V = Vec4<T>;
    constexpr int RZ = G::RZ, LY = G::LY, TZ = G::TZ, TY = G::TY, SW = G::SW;
    constexpr int U = TmaUnroll<R, FORM>::U;
    constexpr int Q = 2 * R + U;  // queue slots: 2R planes of history/lookahead + U fronts
    constexpr int NWIN = 4 + 2 * RZ;  // z window values
    constexpr int S = TmaPipe<R>::STAGES;
    static_assert(YB == 1 || YB == 2, "one or two rows per thread");
    static_assert(YB == 1 || MODE == kModeStep, "two rows per thread: the plain step");
    uint64_t *bars = reinterpret_cast<uint64_t *>(ring - 128);  // placed by tma_ring_init

    const int tid = threadIdx.x;
    const int warp = tid >> 5, lane = tid & 31;
    const int lz = lane % LZ, ly = lane / LZ;
    const int z0 = bz * TZ, y0 = by * TY;
    const int ty = (warp * LY + ly) * YB;  // the thread's first row in the tile
    const int z4 = z0 + 4 * lz;
    const long long P = a.plane;
    bool own[YB];
    const T *u[YB];
    T *up[YB];
    T *un[YB];
#pragma unroll
    for (int r = 0; r < YB; ++r) {
        const int y = y0 + ty + r;
        own[r] = (y < a.Ny) && (z4 < a.Nz);
        const long long col = (long long)y * a.pz + z4;
        u[r] = static_cast<const T *>(a.u) + col;
        up[r] = static_cast<T *>(a.up) + col;  // FP32: u^{n-1} -> u^{n+1}; 16-bit: d^n -> d^{n+1}
        un[r] = Io<T>::kScaled ? static_cast<T *>(a.un) + col : nullptr;  // 16-bit: u^{n+1}
    }
    static_assert(MODE == kModeStep || (FORM == kFactored && !Io<T>::kScaled), "gradient modes: FP32 factored");
    const long long col0 = (long long)(y0 + ty) * a.pz + z4;
    float *hist = MODE != kModeStep ? a.hist + col0 : nullptr;
    float *grad = MODE == kModeAdjointGrad ? a.grad + col0 : nullptr;
    const int g0 = g;
    g += xe - xb;

    // the whole y-z tile lies where the damping field vanishes (in y and z): such planes
    // inside the box's x range need no g tile
    const bool tile_yz_box = y0 >= a.by0 && y0 + TY <= a.by1 && z0 >= a.bz0 && z0 + TZ <= a.bz1;
    // the argument fields the plane loop reads, as scalars: arguments in shared memory
    // (the batch kernels) would otherwise be read again after every memory clobber of
    // the loop's barrier and copy code
    const int a_Nx = a.Nx, a_bx0 = a.bx0, a_bx1 = a.bx1;
    const float a_half_dt = a.half_dt, a_dt2 = a.dt2;
    // the row's points past its end (kept zero: the pitch padding)
    const unsigned tail_mask = (z4 + 1 >= a.Nz ? 2u : 0u) | (z4 + 2 >= a.Nz ? 4u : 0u) | (z4 + 3 >= a.Nz ? 8u : 0u);
    auto g_free = [&](int x) { return tile_yz_box && x >= a_bx0 && x < a_bx1; };
    // every input of plane x arrives in its ring stage by bulk tensor copies
    auto issue = [&](int x, int stage) {
        const uint32_t bar = smem_addr(&bars[stage]);
        unsigned char *st = ring + stage * G::STAGE_BYTES;
        const bool need_g = !g_free(x);
        mbar_expect_tx(bar, uint32_t(G::HALO_RAW + 2 * G::PT_T_RAW +
                                     ((need_g ? 2 : 1) + (MODE == kModeAdjointGrad ? 2 : 0)) * G::PT_F_RAW));
        if constexpr (MODE == kModeAdjointGrad) {
            tma_load_4d(smem_addr(st + G::OFF_X0), &gm->hist, bar, z0, y0, x, a.hist_slot);
            tma_load_3d(smem_addr(st + G::OFF_X1), &gm->grad, bar, z0, y0, x);
        }
        tma_load_3d(smem_addr(st), &maps->u_halo, bar, z0 - RZ, y0 - R, x);
        tma_load_3d(smem_addr(st + G::OFF_FRONT), &maps->u_pt, bar, z0, y0, x + R);  // zero past Nx
        tma_load_3d(smem_addr(st + G::OFF_UP), &maps->up_pt, bar, z0, y0, x);
        tma_load_3d(smem_addr(st + G::OFF_F1), &maps->f1_pt, bar, z0, y0, x);
        if (need_g) tma_load_3d(smem_addr(st + G::OFF_F2), &maps->f2_pt, bar, z0, y0, x);
    };
    auto prefetch = [&](int x) {
        // point data of plane x and the queue front of plane x + R into L2
        if (x < xe) {
            tma_prefetch_3d(&maps->up_pt, z0, y0, x);
            tma_prefetch_3d(&maps->f1_pt, z0, y0, x);
            if (!g_free(x)) tma_prefetch_3d(&maps->f2_pt, z0, y0, x);
            if (x + R < a_Nx) tma_prefetch_3d(&maps->u_pt, z0, y0, x + R);
        }
    };
    if (tid == 0) {
        for (int s = 0; s < S - 1 && xb + s < xe; ++s) issue(xb + s, (g0 + s) % S);
        for (int d = 1; d <= kPrefetchAhead; ++d) prefetch(xb + d);
    }

    // sources among each row's 4 points: bit s set, sub-index in src_p
    unsigned src_mask[YB];
    int src_p[YB][kFusedSources];
#pragma unroll
    for (int r = 0; r < YB; ++r) {
        src_mask[r] = 0;
#pragma unroll
        for (int s = 0; s < kFusedSources; ++s) {
            src_p[r][s] = 0;
            if (own[r] && s < a.ns && a.sy[s] == y0 + ty + r && a.sz[s] >= z4 && a.sz[s] < z4 + 4 &&
                a.sx[s] >= xb && a.sx[s] < xe) {
                src_mask[r] |= 1u << s;
                src_p[r][s] = a.sz[s] - z4;
            }
        }
    }

    const float4 zero4 = make_float4(0.f, 0.f, 0.f, 0.f);
    auto load_u = [&](int r, int x) -> float4 {
        if (!(own[r] && x >= 0 && x < a.Nx)) return zero4;
        if constexpr (COHERENT) {
            return V::ldcg(u[r] + x * P);
        } else {
            return V::ldg(u[r] + x * P);
        }
    };
    float4 q[YB][Q];
#pragma unroll
    for (int r = 0; r < YB; ++r)
#pragma unroll
        for (int k = 0; k < 2 * R; ++k) q[r][k] = load_u(r, xb - R + k);

    float2 cz2[R + 1];
#pragma unroll
    for (int j = 1; j <= R; ++j) cz2[j] = f2(a.coef[j], a.coef[j]);
    // 16-bit storage: every factor below is a power of two, so folding the output
    // scales into the input scales changes no rounding (barring subnormals):
    // d_st = w (L u_raw) s_u/s_d' + (1 - 2g) d_raw s_d/s_d' and
    // u_st = u_raw s_u/s_u' + d_st s_d'/s_u' are the stored (scaled) values directly
    // FP32 storage has no scales: the factor is a compile-time 1 there
    const float kd = Io<T>::kScaled ? sc.inv_s_d_out : 1.0f;
    const float2 su2 = f2(sc.s_u * kd, sc.s_u * kd), sd2 = f2(sc.s_d * kd, sc.s_d * kd);
    const float2 uu2 = f2(sc.s_u * sc.inv_s_out, sc.s_u * sc.inv_s_out);
    const float2 rr2 = f2(sc.s_d_out * sc.inv_s_out, sc.s_d_out * sc.inv_s_out);
    const int colw = 4 * lz;  // first element of the thread's z window in a tile row
    unsigned amax_bits = acc.amax_bits, damax_bits = acc.damax_bits;
    // FP32 storage needs only to know whether a non-finite value was written:
    // v - v is 0 for finite v and NaN otherwise, and NaN persists through the sum
    float2 nonfinite = f2(0.f, 0.f);
    bool over = acc.over;
    bool failed = false;
    int issued = min(S - 1, xe - xb);  // planes handed to the copy engine (tid 0's count)
    int it_failed = 0;                  // first plane whose wait gave up
    int stage = g0 % S;                 // ring stage and mbarrier phase of the current plane
    uint32_t phase = uint32_t(g0 / S) & 1u;
    bool any_own = false;
#pragma unroll
    for (int r = 0; r < YB; ++r) any_own |= own[r];

    for (int xo = xb; xo < xe; xo += U) {
#pragma unroll
        for (int i = 0; i < U; ++i) {
            const int x = xo + i;
            if (x >= xe) break;
            const int it = x - xb;
            const bool ok = mbar_wait_bounded(smem_addr(&bars[stage]), phase);
            if (__syncthreads_or(!ok)) {
                failed = true;
                it_failed = it;
                break;
            }
            if (tid == 0) {
                if (x + S - 1 < xe) {
                    // plane x + S - 1 takes the stage of plane x - 1, which every thread has
                    // finished reading (it passed the barrier above)
                    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
                    issue(x + S - 1, stage == 0 ? S - 1 : stage - 1);
                    ++issued;
                }
                prefetch(x + 1 + kPrefetchAhead);
            }
            const unsigned char *st = ring + stage * G::STAGE_BYTES;
#pragma unroll
            for (int r = 0; r < YB; ++r)
                q[r][2 * R + i] = V::ld(reinterpret_cast<const T *>(st + G::OFF_FRONT) + (ty + r) * TZ + 4 * lz);
            float4 dv, gv;  // adjoint pass: D^{k-1} and the gradient at this plane (from the ring)
            if constexpr (MODE == kModeAdjointGrad) {
                if (own[0]) {
                    const int po = ty * TZ + 4 * lz;
                    dv = *reinterpret_cast<const float4 *>(reinterpret_cast<const float *>(st + G::OFF_X0) + po);
                    gv = *reinterpret_cast<const float4 *>(reinterpret_cast<const float *>(st + G::OFF_X1) + po);
                }
            }
            if (any_own) {
                const T *t = reinterpret_cast<const T *>(st);
                const T *rowp = t + (ty + R) * SW + colw;  // the first row's window in the halo tile
                const bool gf = g_free(x);
                float win[YB][NWIN];
#pragma unroll
                for (int r = 0; r < YB; ++r)
#pragma unroll
                    for (int m = 0; m < NWIN / 4; ++m) {
                        const float4 v = V::ld(rowp + r * SW + 4 * m);
                        win[r][4 * m] = v.x;
                        win[r][4 * m + 1] = v.y;
                        win[r][4 * m + 2] = v.z;
                        win[r][4 * m + 3] = v.w;
                    }
                float4 uc[YB];
#pragma unroll
                for (int r = 0; r < YB; ++r) uc[r] = q[r][R + i];
                // the y taps at distance j of row r: ym(r, j) = row r - j, yp(r, j) = row r + j.
                // Two rows share the loads: iteration j loads rows -j and j + 1 (relative to
                // the first row) and keeps rows j and 1 - j from the previous iteration
                // (iteration 1 takes them from the rows' centres).
                float4 lo_prev = uc[0], hi_prev = uc[YB - 1];
                auto ytaps = [&](int j, float4 *ym, float4 *yp) {
                    if constexpr (YB == 1) {
                        ym[0] = V::ld(rowp + RZ - j * SW);
                        yp[0] = V::ld(rowp + RZ + j * SW);
                    } else {
                        const float4 lo = V::ld(rowp + RZ - j * SW), hi = V::ld(rowp + RZ + (j + 1) * SW);
                        ym[0] = lo;
                        yp[0] = hi_prev;
                        ym[1] = lo_prev;
                        yp[1] = hi;
                        lo_prev = lo;
                        hi_prev = hi;
                    }
                };
                float2 lapA[YB], lapB[YB];
#pragma unroll
                for (int r = 0; r < YB; ++r) lapA[r] = lapB[r] = f2(0.f, 0.f);
                float4 cum[YB], cf1[YB], cf2[YB], out[YB];
#pragma unroll
                for (int r = 0; r < YB; ++r) {
                    const int po = (ty + r) * TZ + 4 * lz;  // the row's 4 points in a point tile
                    cum[r] = V::ld(reinterpret_cast<const T *>(st + G::OFF_UP) + po);
                    cf1[r] = *reinterpret_cast<const float4 *>(reinterpret_cast<const float *>(st + G::OFF_F1) + po);
                    cf2[r] = gf ? zero4
                                : *reinterpret_cast<const float4 *>(reinterpret_cast<const float *>(st + G::OFF_F2) + po);
                }
                float sw[YB][4];
                if constexpr (FORM == kFactored) {
                    // -6 u_c is added to each distance-j sum: exact zero for a constant field
                    float2 nsixA[YB], nsixB[YB];
#pragma unroll
                    for (int r = 0; r < YB; ++r) {
                        nsixA[r] = mul2(f2(-6.f, -6.f), lo2(uc[r]));
                        nsixB[r] = mul2(f2(-6.f, -6.f), hi2(uc[r]));
                    }
#pragma unroll
                    for (int j = 1; j <= R; ++j) {
                        float4 ym[YB], yp[YB];
                        ytaps(j, ym, yp);
#pragma unroll
                        for (int r = 0; r < YB; ++r) {
                            const float4 xm = q[r][R + i - j], xp = q[r][R + i + j];
                            const float2 sA = add2(add2(add2(lo2(xm), lo2(xp)), add2(lo2(ym[r]), lo2(yp[r]))),
                                                   ztap_pair<RZ>(win[r], j));
                            const float2 sB = add2(add2(add2(hi2(xm), hi2(xp)), add2(hi2(ym[r]), hi2(yp[r]))),
                                                   ztap_pair<RZ + 2>(win[r], j));
                            lapA[r] = fma2(cz2[j], add2(sA, nsixA[r]), lapA[r]);
                            lapB[r] = fma2(cz2[j], add2(sB, nsixB[r]), lapB[r]);
                        }
                    }
#pragma unroll
                    for (int r = 0; r < YB; ++r) {
                        if constexpr (Io<T>::kScaled) {
                            // increment form: d+ = w L u + (1 - 2g) d, u+ = u + d+ (formed below,
                            // after the source), directly in the output scales; where the damping
                            // vanishes 1 - 2g is exactly 1
                            const float2 lA = mul2(lapA[r], su2), lB = mul2(lapB[r], su2);
                            float2 pA = mul2(lo2(cum[r]), sd2), pB = mul2(hi2(cum[r]), sd2);
                            if (!gf) {
                                pA = mul2(fma2(f2(-2.f, -2.f), lo2(cf2[r]), f2(1.f, 1.f)), pA);
                                pB = mul2(fma2(f2(-2.f, -2.f), hi2(cf2[r]), f2(1.f, 1.f)), pB);
                            }
                            const float2 dA = fma2(lo2(cf1[r]), lA, pA);
                            const float2 dB = fma2(hi2(cf1[r]), lB, pB);
                            out[r] = make_float4(dA.x, dA.y, dB.x, dB.y);
                        } else {
                            // u+ = w L + (2u - u-) - 2 g (u - u-); the last term only where the
                            // damping does not vanish
                            const float2 ucA = lo2(uc[r]), ucB = hi2(uc[r]), umA = lo2(cum[r]), umB = hi2(cum[r]);
                            const float2 dA = fma2(f2(-1.f, -1.f), umA, ucA), dB = fma2(f2(-1.f, -1.f), umB, ucB);
                            float2 vA = fma2(lo2(cf1[r]), lapA[r], add2(ucA, dA));
                            float2 vB = fma2(hi2(cf1[r]), lapB[r], add2(ucB, dB));
                            if (!gf) {
                                vA = fma2(mul2(f2(-2.f, -2.f), lo2(cf2[r])), dA, vA);
                                vB = fma2(mul2(f2(-2.f, -2.f), hi2(cf2[r])), dB, vB);
                            }
                            out[r] = make_float4(vA.x, vA.y, vB.x, vB.y);
                        }
                        sw[r][0] = cf1[r].x * kd;  // kd = 1 for FP32 storage
                        sw[r][1] = cf1[r].y * kd;
                        sw[r][2] = cf1[r].z * kd;
                        sw[r][3] = cf1[r].w * kd;
                    }
                } else {
                    // expanded: every tap (u_tap - u_c) times (c_j dt^2/h^2)/r0
                    static_assert(!Io<T>::kScaled, "16-bit storage uses the factored form");
                    float inv[YB][4];
                    float2 invA[YB], invB[YB], r0A[YB], r0B[YB];
#pragma unroll
                    for (int r = 0; r < YB; ++r) {
                        // r0 = m + dt/2 eta, two points per instruction
                        const float2 hdt = f2(a_half_dt, a_half_dt);
                        r0A[r] = fma2(hdt, lo2(cf2[r]), lo2(cf1[r]));
                        r0B[r] = fma2(hdt, hi2(cf2[r]), hi2(cf1[r]));
                        inv[r][0] = expanded_inv(r0A[r].x);
                        inv[r][1] = expanded_inv(r0A[r].y);
                        inv[r][2] = expanded_inv(r0B[r].x);
                        inv[r][3] = expanded_inv(r0B[r].y);
                        invA[r] = f2(inv[r][0], inv[r][1]);
                        invB[r] = f2(inv[r][2], inv[r][3]);
                    }
#pragma unroll
                    for (int j = 1; j <= R; ++j) {
                        float4 ym[YB], yp[YB];
                        ytaps(j, ym, yp);
#pragma unroll
                        for (int r = 0; r < YB; ++r) {
                            const float4 xm = q[r][R + i - j], xp = q[r][R + i + j];
                            const float2 ucA = lo2(uc[r]), ucB = hi2(uc[r]);
                            const float *w = win[r];
                            const float2 cA = mul2(cz2[j], invA[r]), cB = mul2(cz2[j], invB[r]);
                            lapA[r] = fma2(cA, sub2(lo2(xm), ucA), lapA[r]);
                            lapA[r] = fma2(cA, sub2(lo2(xp), ucA), lapA[r]);
                            lapA[r] = fma2(cA, sub2(lo2(ym[r]), ucA), lapA[r]);
                            lapA[r] = fma2(cA, sub2(lo2(yp[r]), ucA), lapA[r]);
                            lapA[r] = fma2(cA, zdiff_pair<RZ>(w, -j, ucA), lapA[r]);
                            lapA[r] = fma2(cA, zdiff_pair<RZ>(w, j, ucA), lapA[r]);
                            lapB[r] = fma2(cB, sub2(hi2(xm), ucB), lapB[r]);
                            lapB[r] = fma2(cB, sub2(hi2(xp), ucB), lapB[r]);
                            lapB[r] = fma2(cB, sub2(hi2(ym[r]), ucB), lapB[r]);
                            lapB[r] = fma2(cB, sub2(hi2(yp[r]), ucB), lapB[r]);
                            lapB[r] = fma2(cB, zdiff_pair<RZ + 2>(w, -j, ucB), lapB[r]);
                            lapB[r] = fma2(cB, zdiff_pair<RZ + 2>(w, j, ucB), lapB[r]);
                        }
                    }
#pragma unroll
                    for (int r = 0; r < YB; ++r) {
                        // u+ = L + (2a) u + (1 - 2a) u-, a = m / r0 by a correctly rounded
                        // division; where the damping vanishes (the tile's plane inside the
                        // undamped box) r0 = m exactly and a = 1, so the level coefficients are
                        // the constants 2 and -1
                        float2 vA, vB;
                        if (gf) {
                            vA = fma2(f2(-1.f, -1.f), lo2(cum[r]), fma2(f2(2.f, 2.f), lo2(uc[r]), lapA[r]));
                            vB = fma2(f2(-1.f, -1.f), hi2(cum[r]), fma2(f2(2.f, 2.f), hi2(uc[r]), lapB[r]));
                        } else {
                            const float am[4] = {__fdiv_rn(cf1[r].x, r0A[r].x), __fdiv_rn(cf1[r].y, r0A[r].y),
                                                 __fdiv_rn(cf1[r].z, r0B[r].x), __fdiv_rn(cf1[r].w, r0B[r].y)};
                            vA = fma2(f2(1.0f - 2.0f * am[0], 1.0f - 2.0f * am[1]), lo2(cum[r]),
                                      fma2(f2(2.0f * am[0], 2.0f * am[1]), lo2(uc[r]), lapA[r]));
                            vB = fma2(f2(1.0f - 2.0f * am[2], 1.0f - 2.0f * am[3]), hi2(cum[r]),
                                      fma2(f2(2.0f * am[2], 2.0f * am[3]), hi2(uc[r]), lapB[r]));
                        }
                        if (src_mask[r]) {  // source weights dt^2 / r0, only where a source sits
#pragma unroll
                            for (int p = 0; p < 4; ++p) sw[r][p] = a_dt2 * inv[r][p];
                        }
                        out[r] = make_float4(vA.x, vA.y, vB.x, vB.y);
                    }
                }
#pragma unroll
                for (int r = 0; r < YB; ++r) {
                    if (!own[r]) continue;
                    float4 o = out[r];
                    if (src_mask[r]) {
#pragma unroll
                        for (int s = 0; s < kFusedSources; ++s) {
                            if (((src_mask[r] >> s) & 1u) && a.sx[s] == x) {
                                const float qv = step < 0 ? source_value(a, s)
                                                          : step < a.ld ? __ldg(a.wavelet + (long long)s * a.ld + step)
                                                                        : 0.0f;
                                const int p = src_p[r][s];
                                if (p == 0) o.x = fmaf(sw[r][0], qv, o.x);
                                if (p == 1) o.y = fmaf(sw[r][1], qv, o.y);
                                if (p == 2) o.z = fmaf(sw[r][2], qv, o.z);
                                if (p == 3) o.w = fmaf(sw[r][3], qv, o.w);
                            }
                        }
                    }
                    if (tail_mask) {  // row tail: keep the pitch padding zero
                        if (tail_mask & 2u) o.y = 0.f;
                        if (tail_mask & 4u) o.z = 0.f;
                        if (tail_mask & 8u) o.w = 0.f;
                    }
                    auto bits4 = [](const float4 &v) {
                        return max(max(__float_as_uint(fabsf(v.x)), __float_as_uint(fabsf(v.y))),
                                   max(__float_as_uint(fabsf(v.z)), __float_as_uint(fabsf(v.w))));
                    };
                    if constexpr (Io<T>::kScaled) {
                        // o is the stored d^{n+1}; u^{n+1} = u^n + d^{n+1}, stored (padding
                        // stays zero: both terms are). The maxima are of stored values (scaled
                        // back once, after the loop); the 16-bit range is checked there too.
                        const float2 nA = fma2(lo2(uc[r]), uu2, mul2(f2(o.x, o.y), rr2));
                        const float2 nB = fma2(hi2(uc[r]), uu2, mul2(f2(o.z, o.w), rr2));
                        const float4 unew = make_float4(nA.x, nA.y, nB.x, nB.y);
                        damax_bits = max(damax_bits, bits4(o));
                        amax_bits = max(amax_bits, bits4(unew));
                        V::st(un[r] + x * P, unew);
                    } else {
                        // x * 0 is 0 for finite x and NaN otherwise
                        nonfinite = fma2(f2(o.x, o.y), f2(0.f, 0.f), nonfinite);
                        nonfinite = fma2(f2(o.z, o.w), f2(0.f, 0.f), nonfinite);
                    }
                    V::st(up[r] + x * P, o);
                    if constexpr (MODE == kModeForwardD) {
                        // D = (u^{n+1} - 2u^n) + u^{n-1}; FP32 factored: cum is u^{n-1}
                        const float4 d4 = make_float4(fmaf(-2.0f, uc[r].x, o.x) + cum[r].x,
                                                      fmaf(-2.0f, uc[r].y, o.y) + cum[r].y,
                                                      fmaf(-2.0f, uc[r].z, o.z) + cum[r].z,
                                                      fmaf(-2.0f, uc[r].w, o.w) + cum[r].w);
                        __stcs(reinterpret_cast<float4 *>(hist + x * P), d4);
                    }
                    if constexpr (MODE == kModeAdjointGrad) {
                        gv = make_float4(fmaf(-o.x, dv.x, gv.x), fmaf(-o.y, dv.y, gv.y), fmaf(-o.z, dv.z, gv.z),
                                         fmaf(-o.w, dv.w, gv.w));
                        *reinterpret_cast<float4 *>(grad + x * P) = gv;
                    }
                }
            }
            if (++stage == S) {
                stage = 0;
                phase ^= 1u;
            }
        }
        if (failed) break;
#pragma unroll
        for (int r = 0; r < YB; ++r)
#pragma unroll
            for (int k = 0; k < 2 * R; ++k) q[r][k] = q[r][k + U];
    }
    if (failed) {
        // planes it_failed .. issued-1 are the only copies not yet waited for (one per stage)
        if (tid == 0) {
            if (a.status) atomicOr(a.status, kStatusTimeout);
            for (int it = it_failed; it < issued; ++it)
                mbar_wait_bounded(smem_addr(&bars[(g0 + it) % S]), uint32_t((g0 + it) / S) & 1u);
        }
        return false;
    }
    if constexpr (!Io<T>::kScaled) {
        // as bits: NaN sorts above every finite magnitude (the status test)
        if (!(nonfinite.x == 0.f && nonfinite.y == 0.f)) amax_bits = 0x7fc00000u;
    }
    acc.amax_bits = amax_bits;
    acc.damax_bits = damax_bits;
    acc.over = over;
    return true;
}

// 16-bit storage: the per-thread maxima were taken over stored (scaled) values;
// check them against the format's range and scale them back to true values
// (powers of two: exact) for the next level's scale selection.
template <typename T>
__device__ __forceinline__ void tma_finish(TmaAcc &acc, const ScaleState &sc) {
    if constexpr (Io<T>::kScaled) {
        const float dmax = __uint_as_float(acc.damax_bits), umax = __uint_as_float(acc.amax_bits);
        acc.over |= dmax > Io<T>::kMaxStored || umax > Io<T>::kMaxStored;
        acc.damax_bits = __float_as_uint(dmax * sc.s_d_out);
        acc.amax_bits = __float_as_uint(umax * sc.s_out);
    }
}

// Receivers of a single-shot step: every thread of the grid samples at most a
// few receivers from the step's input level u^n (read-only during the step),
// trilinear, corners summed in a fixed order and dequantised with the level's
// scale, as the standalone sampling kernel does (same values bit for bit).
template <typename T>
__device__ __forceinline__ void tma_sample_receivers(const StepArgs &a, float scale) {
    const long long nthreads = (long long)gridDim.x * gridDim.y * gridDim.z * blockDim.x;
    const long long cta = blockIdx.x + (long long)gridDim.x * (blockIdx.y + (long long)gridDim.y * blockIdx.z);
    const T *u = static_cast<const T *>(a.u);
    for (long long r = cta * blockDim.x + threadIdx.x; r < a.n_rec; r += nthreads) {
        float v = 0.0f;
#pragma unroll
        for (int c = 0; c < 8; ++c) v = fmaf(a.rec_w[8 * r + c], Io<T>::to_f(u[a.rec_off[8 * r + c]]), v);
        a.traces[r * a.rec_stride + a.rec_sample] = Io<T>::kScaled ? v * scale : v;
    }
}

// Single-shot step: CTA (bz, by, bx) streams planes [bx x_block, (bx+1) x_block)
// of tile (bz, by). The grid runs z-tiles fastest and x-chunks slowest, so the
// CTAs resident at any moment cover neighbouring tiles at the same planes and
// share their halo rows in L2.
template <int R, int FORM, int LZ, int W, typename T, int YB = 1>
__global__ void __launch_bounds__(32 * W, (tma_warps_per_sm(R, YB) / W > 0 ? tma_warps_per_sm(R, YB) / W : 1))
    fd_tma_kernel(const __grid_constant__ TmaMaps maps, const StepArgs a, int check) {
    extern __shared__ __align__(128) unsigned char smem_dyn[];
    publish_scales<T>(a, blockIdx.x == 0 && blockIdx.y == 0 && blockIdx.z == 0 && threadIdx.x == 0);
    unsigned char *ring = tma_ring_init<R>(smem_dyn);
    const ScaleState sc = read_scales<T>(a);
    if (a.rec_sample >= 0 && a.n_rec > 0) tma_sample_receivers<T>(a, sc.s_u);
    const int xb = a.x_lo + blockIdx.z * a.x_block;
    int g = 0;
    TmaAcc acc;
    if (tma_segment<R, FORM, LZ, W, T, kModeStep, false, YB>(&maps, a, sc, blockIdx.x, blockIdx.y, xb,
                                                            min(xb + a.x_block, a.x_hi), ring, g, acc) &&
        check) {
        tma_finish<T>(acc, sc);
        reduce_amax(a, acc.amax_bits, acc.over, acc.damax_bits);
    }
}

// The FWI gradient's passes (FP32 factored; sources and receivers as the step).
template <int R, int LZ, int W, int MODE>
__global__ void __launch_bounds__(32 * W, (tma_warps_per_sm(R) / W > 0 ? tma_warps_per_sm(R) / W : 1)) fd_tma_grad_kernel(const __grid_constant__ TmaMaps maps,
                                                             const __grid_constant__ GradMaps gmaps,
                                                             const StepArgs a, int check) {
    extern __shared__ __align__(128) unsigned char smem_dyn[];
    unsigned char *ring = tma_ring_init<R>(smem_dyn);
    const ScaleState sc = read_scales<float>(a);
    if (a.rec_sample >= 0 && a.n_rec > 0) tma_sample_receivers<float>(a, 1.0f);
    const int xb = blockIdx.z * a.x_block;
    int g = 0;
    TmaAcc acc;
    if (tma_segment<R, kFactored, LZ, W, float, MODE>(&maps, a, sc, blockIdx.x, blockIdx.y, xb,
                                                      min(xb + a.x_block, a.Nx), ring, g, acc, &gmaps) &&
        check)
        reduce_amax(a, acc.amax_bits, acc.over, acc.damax_bits);
}

template <int R, int LZ, int W, int MODE>
cudaError_t tma_grad_launch(const TmaMaps &maps, const GradMaps &gm, const StepArgs &a, bool check, cudaStream_t s) {
    using G = TmaShape<R, LZ, W, float, MODE == kModeAdjointGrad ? 2 : 0>;
    auto kernel = fd_tma_grad_kernel<R, LZ, W, MODE>;
    static bool attr_set = false;
    if (!attr_set) {
        cudaError_t e = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, G::SMEM_BYTES);
        if (e != cudaSuccess) return e;
        attr_set = true;
    }
    const dim3 grid((a.Nz + G::TZ - 1) / G::TZ, (a.Ny + G::TY - 1) / G::TY, (a.Nx + a.x_block - 1) / a.x_block);
    kernel<<<grid, 32 * W, G::SMEM_BYTES, s>>>(maps, gm, a, check ? 1 : 0);
    return cudaGetLastError();
}

// Gradient passes exist for the 32x16 tile (LZ 8, W 4) only.
template <int R>
cudaError_t tma_grad_step_r(int mode, const TmaMaps &map, const GradMaps &gm, const StepArgs &a, bool check,
                            cudaStream_t s) {
    if (mode == kModeForwardD) return tma_grad_launch<R, 8, 4, kModeForwardD>(map, gm, a, check, s);
    if (mode == kModeAdjointGrad) return tma_grad_launch<R, 8, 4, kModeAdjointGrad>(map, gm, a, check, s);
    return cudaErrorInvalidValue;
}

template <int R, int FORM, int LZ, int W, typename T, int YB = 1>
cudaError_t tma_launch(const TmaMaps &maps, const StepArgs &a, bool check, cudaStream_t s) {
    using G = TmaShape<R, LZ, W, T, 0, YB>;
    auto kernel = fd_tma_kernel<R, FORM, LZ, W, T, YB>;
    static bool attr_set = false;  // per instantiation, set once per process
    if (!attr_set) {
        cudaError_t e = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, G::SMEM_BYTES);
        if (e != cudaSuccess) return e;
        attr_set = true;
    }
    if (a.x_hi <= a.x_lo) return cudaSuccess;  // no planes to update
    const dim3 grid((a.Nz + G::TZ - 1) / G::TZ, (a.Ny + G::TY - 1) / G::TY,
                    (a.x_hi - a.x_lo + a.x_block - 1) / a.x_block);
    kernel<<<grid, 32 * W, G::SMEM_BYTES, s>>>(maps, a, check ? 1 : 0);
    return cudaGetLastError();
}

// Batched form: one CTA per work item (shot, bz, by, bx) of a device table, so
// many uneven shots advance in one launch. Each CTA copies its shot's step
// arguments into shared memory (with the step index of this launch) and runs
// one segment (planes [bx x_block, (bx+1) x_block) of tile (bz, by)) of the
// single-shot kernel's schedule.
template <int R, int FORM, int LZ, int W, typename T>
__global__ void __launch_bounds__(32 * W, (tma_warps_per_sm(R) / W > 0 ? tma_warps_per_sm(R) / W : 1)) fd_tma_batch_kernel(const BatchShot *__restrict__ shots,
                                                              const int4 *__restrict__ items, int offset) {
    extern __shared__ __align__(128) unsigned char smem_dyn[];
    __shared__ StepArgs sa;
    const int4 it = items[blockIdx.x];  // (shot, bz, by, bx)
    const BatchShot &sh = shots[it.x];
    const int p = (sh.cur0 + offset) & 1;
    const TmaMaps *maps = &sh.maps[p];
    if (threadIdx.x == 0) {
        sa = sh.args[p];
        sa.step = sh.step0 + offset;
        // the maps were written to global memory by the host: acquire them for the copy engine
        const CUtensorMap *m[5] = {&maps->u_halo, &maps->u_pt, &maps->up_pt, &maps->f1_pt, &maps->f2_pt};
#pragma unroll
        for (int k = 0; k < 5; ++k)
            asm volatile("fence.proxy.tensormap::generic.acquire.gpu [%0], 128;" ::"l"(
                             reinterpret_cast<uint64_t>(m[k]))
                         : "memory");
    }
    __syncthreads();
    publish_scales<T>(sa, it.y == 0 && it.z == 0 && it.w == 0 && threadIdx.x == 0);
    unsigned char *ring = tma_ring_init<R>(smem_dyn);
    const ScaleState sc = read_scales<T>(sa);
    const int xb = it.w * sa.x_block;
    int g = 0;
    TmaAcc acc;
    if (tma_segment<R, FORM, LZ, W, T>(maps, sa, sc, it.y, it.z, xb, min(xb + sa.x_block, sa.Nx), ring, g, acc)) {
        tma_finish<T>(acc, sc);
        reduce_amax(sa, acc.amax_bits, acc.over, acc.damax_bits);
    }
}

template <int R, int FORM, int LZ, int W, typename T>
cudaError_t tma_batch_launch(const BatchShot *shots, const int4 *items, int n_items, int offset, cudaStream_t s) {
    using G = TmaShape<R, LZ, W, T>;
    auto kernel = fd_tma_batch_kernel<R, FORM, LZ, W, T>;
    static bool attr_set = false;
    if (!attr_set) {
        cudaError_t e = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, G::SMEM_BYTES);
        if (e != cudaSuccess) return e;
        attr_set = true;
    }
    if (n_items <= 0) return cudaSuccess;
    kernel<<<n_items, 32 * W, G::SMEM_BYTES, s>>>(shots, items, offset);
    return cudaGetLastError();
}

template <int R>
cudaError_t tma_batch_step_r(int form, int storage, int tile_z, int tile_y, const BatchShot *shots,
                             const int4 *items, int n_items, int offset, cudaStream_t s) {
    if constexpr (R > kMaxBatchRadius) {
        return cudaErrorInvalidValue;  // batches stop at space order 16
    } else {
#define FDGB_BATCH_CASE(LZ, W)                                                                          \
    if (tile_z == 4 * (LZ) && tile_y == (32 / (LZ)) * (W)) {                                            \
        if (storage == kF32)                                                                            \
            return form == kFactored ? tma_batch_launch<R, kFactored, LZ, W, float>(shots, items, n_items, offset, s) \
                                     : tma_batch_launch<R, kExpanded, LZ, W, float>(shots, items, n_items, offset, s); \
        if (form == kFactored && storage == kBF16)                                                      \
            return tma_batch_launch<R, kFactored, LZ, W, __nv_bfloat16>(shots, items, n_items, offset, s); \
        if (form == kFactored && storage == kF16)                                                       \
            return tma_batch_launch<R, kFactored, LZ, W, __half>(shots, items, n_items, offset, s);    \
    }
    FDGB_BATCH_CASE(8, 4)
    FDGB_BATCH_CASE(16, 4)
#undef FDGB_BATCH_CASE
    return cudaErrorInvalidValue;
    }
}

// Tile configurations (tile_z, tile_y) of the TMA kernel: (LZ, W) pairs. FP32
// storage has every shape and both forms; 16-bit storage the factored form in
// the shapes of the second list. Above radius 8 (space orders 18-24) the tiles
// are 32 points wide (the widest z window) and the lists shorter.
#define FDGB_TMA_CONFIGS(X) X(8, 8) X(16, 8) X(32, 8) X(8, 4) X(16, 4)
#define FDGB_TMA_CONFIGS_16(X) X(8, 4) X(16, 4)
#define FDGB_TMA_CONFIGS_HIGH(X) X(8, 8) X(8, 4)
#define FDGB_TMA_CONFIGS_16_HIGH(X) X(8, 4)
// Two y rows per thread (radius <= 8, every storage; the factored form for 16-bit):
// 32x32 and 64x16 tiles of 128 threads.
#define FDGB_TMA_CONFIGS2(X) X(8, 4) X(16, 4)

template <int R>
cudaError_t tma_step_r(int form, int storage, int tile_z, int tile_y, int rows, const TmaMaps &map,
                       const StepArgs &a, bool check, cudaStream_t s) {
#define FDGB_TMA_CASE(LZ, W)                                                                    \
    if (storage == kF32 && tile_z == 4 * (LZ) && tile_y == (32 / (LZ)) * (W))                   \
        return form == kFactored ? tma_launch<R, kFactored, LZ, W, float>(map, a, check, s)     \
                                 : tma_launch<R, kExpanded, LZ, W, float>(map, a, check, s);
#define FDGB_TMA_CASE16(LZ, W)                                                                  \
    if (form == kFactored && tile_z == 4 * (LZ) && tile_y == (32 / (LZ)) * (W)) {               \
        if (storage == kBF16) return tma_launch<R, kFactored, LZ, W, __nv_bfloat16>(map, a, check, s); \
        if (storage == kF16) return tma_launch<R, kFactored, LZ, W, __half>(map, a, check, s);  \
    }
#define FDGB_TMA_CASE2(LZ, W)                                                                   \
    if (tile_z == 4 * (LZ) && tile_y == 2 * (32 / (LZ)) * (W)) {                                \
        if (storage == kF32)                                                                    \
            return form == kFactored ? tma_launch<R, kFactored, LZ, W, float, 2>(map, a, check, s) \
                                     : tma_launch<R, kExpanded, LZ, W, float, 2>(map, a, check, s); \
        if (form == kFactored && storage == kBF16)                                              \
            return tma_launch<R, kFactored, LZ, W, __nv_bfloat16, 2>(map, a, check, s);         \
        if (form == kFactored && storage == kF16)                                               \
            return tma_launch<R, kFactored, LZ, W, __half, 2>(map, a, check, s);                \
    }
    if (rows == 2) {
        if constexpr (R <= 8) {
            FDGB_TMA_CONFIGS2(FDGB_TMA_CASE2)
        }
        return cudaErrorInvalidValue;
    }
    if (rows != 1) return cudaErrorInvalidValue;
    if constexpr (R <= 8) {
        FDGB_TMA_CONFIGS(FDGB_TMA_CASE)
        FDGB_TMA_CONFIGS_16(FDGB_TMA_CASE16)
    } else {
        FDGB_TMA_CONFIGS_HIGH(FDGB_TMA_CASE)
        FDGB_TMA_CONFIGS_16_HIGH(FDGB_TMA_CASE16)
    }
#undef FDGB_TMA_CASE
#undef FDGB_TMA_CASE16
#undef FDGB_TMA_CASE2
    return cudaErrorInvalidValue;
}

// Box geometry the host needs to encode the tensor map for a configuration
// (false when the configuration does not exist).
template <int R>
bool tma_box_r(int form, int storage, int tile_z, int tile_y, int rows, int *box_w, int *box_h, int *rz) {
#define FDGB_TMA_BOX_T(LZ, W, T, YB)                                                            \
    {                                                                                           \
        *box_w = TmaShape<R, LZ, W, T, 0, YB>::SW;                                              \
        *box_h = TmaShape<R, LZ, W, T, 0, YB>::SH;                                              \
        *rz = TmaShape<R, LZ, W, T, 0, YB>::RZ;                                                 \
        return true;                                                                            \
    }
#define FDGB_TMA_BOX(LZ, W)                                                                     \
    if (storage == kF32 && tile_z == 4 * (LZ) && tile_y == (32 / (LZ)) * (W)) FDGB_TMA_BOX_T(LZ, W, float, 1)
#define FDGB_TMA_BOX16(LZ, W)                                                                   \
    if (storage != kF32 && form == kFactored && tile_z == 4 * (LZ) && tile_y == (32 / (LZ)) * (W)) \
        FDGB_TMA_BOX_T(LZ, W, __half, 1)
#define FDGB_TMA_BOX2(LZ, W)                                                                    \
    if (tile_z == 4 * (LZ) && tile_y == 2 * (32 / (LZ)) * (W)) {                                \
        if (storage == kF32) FDGB_TMA_BOX_T(LZ, W, float, 2)                                    \
        if (form == kFactored) FDGB_TMA_BOX_T(LZ, W, __half, 2)                                 \
    }
    if (rows == 2) {
        if constexpr (R <= 8) {
            FDGB_TMA_CONFIGS2(FDGB_TMA_BOX2)
        }
        return false;
    }
    if (rows != 1) return false;
    if constexpr (R <= 8) {
        FDGB_TMA_CONFIGS(FDGB_TMA_BOX)
        FDGB_TMA_CONFIGS_16(FDGB_TMA_BOX16)
    } else {
        FDGB_TMA_CONFIGS_HIGH(FDGB_TMA_BOX)
        FDGB_TMA_CONFIGS_16_HIGH(FDGB_TMA_BOX16)
    }
#undef FDGB_TMA_BOX_T
#undef FDGB_TMA_BOX
#undef FDGB_TMA_BOX16
#undef FDGB_TMA_BOX2
    return false;
}

}  // namespace fdgb

#define FDGB_INSTANTIATE_TMA_RADIUS(R)                                                            \
    namespace fdgb {                                                                              \
    cudaError_t tma_step_radius_##R(int form, int storage, int tile_z, int tile_y, int rows,      \
                                    const TmaMaps &map, const StepArgs &a, bool check,            \
                                    cudaStream_t s) {                                             \
        return tma_step_r<R>(form, storage, tile_z, tile_y, rows, map, a, check, s);              \
    }                                                                                             \
    bool tma_box_radius_##R(int form, int storage, int tile_z, int tile_y, int rows, int *w,      \
                            int *h, int *rz) {                                                    \
        return tma_box_r<R>(form, storage, tile_z, tile_y, rows, w, h, rz);                       \
    }                                                                                             \
    cudaError_t tma_batch_step_radius_##R(int form, int storage, int tile_z, int tile_y,          \
                                          const BatchShot *shots, const int4 *items, int n_items, \
                                          int offset, cudaStream_t s) {                           \
        return tma_batch_step_r<R>(form, storage, tile_z, tile_y, shots, items, n_items, offset, s); \
    }                                                                                             \
    cudaError_t tma_grad_step_radius_##R(int mode, const TmaMaps &map, const GradMaps &gm,          \
                                         const StepArgs &a, bool check, cudaStream_t s) {         \
        return tma_grad_step_r<R>(mode, map, gm, a, check, s);                                    \
    }                                                                                             \
    }
