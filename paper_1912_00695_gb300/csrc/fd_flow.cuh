// Flow schedule: one persistent launch advances nt time steps of a shot with
// the single-step kernel's per-point arithmetic and ring (tma_segment), with
// no grid-wide barrier between steps. Work items (step s, x-chunk bx, tile
// by, tile bz), numbered step-major with z fastest, are claimed from a global
// counter. An item of step s > 0 first waits until the 27 items of step s - 1
// around it (x-chunks bx-1..bx+1, tiles by-1..by+1 and bz-1..bz+1) are done:
// they wrote the u^s it reads (halo rows, queue planes, front planes) and they
// were the last readers of the u^{s-1} it overwrites. Every dependency has a
// lower item number, so it was claimed earlier by a running CTA: the waits
// always end (and are bounded all the same). A launch of the per-step
// schedule ends with a tail in which SMs idle while the last CTAs finish, and
// the next launch starts after a gap; here the next step's items fill them.
//
// Memory ordering: the producer's threads store u^{s+1}, the CTA barrier
// orders those stores before thread 0's release store of the item's flag;
// a consumer's thread 0 acquires the flags, orders the copy engine's reads
// after them (proxy fence) and the CTA barrier orders the other threads'
// loads; the queue prologue reads u^s with L1-bypassing loads, since the
// same buffer held older levels earlier in the launch.
//
// The batch flow (fd_tma_batch_flow_kernel, below) applies the same schedule to
// every shot of a batch, with each shot's arguments and tensor maps read from
// device tables instead of the launch's parameters.
#pragma once

#include <type_traits>

#include "fd_flow.h"
#include "fd_tma.cuh"

namespace fdgb {

constexpr unsigned long long kFlowWaitNs = 2000000000ull;  // a dependency wait gives up after 2 s
constexpr long long kFlowWaitLimit = 1LL << 26;            // and after this many polls in any case

__device__ __forceinline__ unsigned ld_acquire_u32(const unsigned *p) {
    unsigned v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

__device__ __forceinline__ void st_release_u32(unsigned *p, unsigned v) {
    asm volatile("st.release.gpu.global.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

// Waits until *flag >= need; false if the wait gave up (kFlowWaitNs of the global
// timer) or the launch aborted.
__device__ __forceinline__ bool flow_wait(const unsigned *flag, unsigned need, const unsigned *abort) {
    unsigned long long t0 = 0;
    for (long long i = 0; i < kFlowWaitLimit; ++i) {
        if (ld_acquire_u32(flag) >= need) return true;
        if (*reinterpret_cast<const volatile unsigned *>(abort)) return false;
        if (i >= 4) {
            if (i == 4) t0 = global_ns();
            else if (global_ns() - t0 > kFlowWaitNs) return false;
            __nanosleep(100);
        }
    }
    return false;
}

// Scales of a flow launch's step s: FP32 none; BF16 the stored levels' own scales
// for the first step's inputs and unit scales otherwise (every level the launch
// writes is stored unscaled: BF16 rounding does not depend on a power-of-two scale).
template <typename T>
__device__ __forceinline__ ScaleState flow_scales(const FlowArgs &f, bool first) {
    ScaleState st{1.0f, 1.0f, 1.0f, 1.0f, 1.0f, 1.0f, 1.0f};
    if constexpr (Io<T>::kScaled) {
        if (first) {
            const int n = level_slot(f.step0);
            st.s_u = f.a[0].scales->scale[n];
            st.s_d = f.a[0].scales->dscale[n];
        }
    }
    return st;
}

// Receivers of the item of step s (FP32): entries [i0, i1) of the region's
// list. Each receiver's other corners lie in the neighbouring regions, whose
// u^{step0+s} the dependency wait has seen completed and which no item
// overwrites before this item's flag. An entry holds the pitched offset of the
// lower corner node; corner c = 4 dx + 2 dy + dz sits at that offset plus
// dx plane + dy pz + dz, the node the receiver's own table names, and the
// corners are summed in that order as the single-step kernel sums them (same
// bits). A thread takes kRecBatch entries at a time so that their loads are in
// flight together; the field loads bypass L1, since the buffer held older
// levels earlier in the launch. Kept out of line: the kernel variant's
// register allocation stays that of the plain flow.
constexpr int kRecBatch = 1;
static __device__ __noinline__ void flow_sample_receivers(const FlowArgs &f, const StepArgs &a, int s, int i0,
                                                          int i1) {
    const long long smp = f.step0 + s - f.rec_s0 - 1;
    if (smp < 0 || smp >= f.rec_stride) return;
    const float *__restrict__ u = static_cast<const float *>(a.u);
    const long long dxy[4] = {0, a.pz, a.plane, a.plane + a.pz};
    const int nthr = int(blockDim.x);
    for (int i = i0 + int(threadIdx.x); i < i1; i += kRecBatch * nthr) {
        long long base[kRecBatch];
        float w[kRecBatch][8], c[kRecBatch][8];
        int row[kRecBatch];
#pragma unroll
        for (int b = 0; b < kRecBatch; ++b) {
            const int e = i + b * nthr;
            if (e < i1) {
                base[b] = __ldg(f.rec_off + e);
                row[b] = __ldg(f.rec_row + e);
                const float4 *wp = reinterpret_cast<const float4 *>(f.rec_w) + 2 * (long long)e;
                const float4 w03 = __ldg(wp), w47 = __ldg(wp + 1);
                w[b][0] = w03.x, w[b][1] = w03.y, w[b][2] = w03.z, w[b][3] = w03.w;
                w[b][4] = w47.x, w[b][5] = w47.y, w[b][6] = w47.z, w[b][7] = w47.w;
            }
        }
#pragma unroll
        for (int b = 0; b < kRecBatch; ++b)
            if (i + b * nthr < i1) {
#pragma unroll
                for (int k = 0; k < 8; ++k) c[b][k] = __ldcg(u + base[b] + dxy[((k >> 2) << 1) | ((k >> 1) & 1)] + (k & 1));
            }
#pragma unroll
        for (int b = 0; b < kRecBatch; ++b)
            if (i + b * nthr < i1) {
                float v = 0.0f;
#pragma unroll
                for (int k = 0; k < 8; ++k) v = fmaf(w[b][k], c[b][k], v);
                f.traces[(long long)row[b] * f.rec_stride + smp] = v;
            }
    }
}

// Sources beyond the fused ones, item of step s (FP32): entries [i0, i1) of the
// region's list, added after the item's stores of u^{step0+s+1} and before its
// flag, as the per-step extra-source kernel adds them (one thread per entry at
// distinct nodes, else one thread in source order).
static __device__ __noinline__ void flow_inject_extra(const FlowArgs &f, const StepArgs &a, int s, int i0, int i1,
                                                      bool expanded) {
    const long long step = f.step0 + s;
    if (step < 0 || step >= a.ld) return;
    float *up = static_cast<float *>(a.up);
    const int t = int(threadIdx.x);
    if (!f.xs_distinct) {
        if (t != 0) return;
        for (int i = i0; i < i1; ++i) {
            const long long p = f.xs_off[i];
            add_extra_source_f32(up, p, extra_source_weight(a, p, expanded), a.wavelet[(long long)f.xs_idx[i] * a.ld + step]);
        }
        return;
    }
    for (int i = i0 + t; i < i1; i += int(blockDim.x)) {
        const long long p = f.xs_off[i];
        add_extra_source_f32(up, p, extra_source_weight(a, p, expanded), a.wavelet[(long long)f.xs_idx[i] * a.ld + step]);
    }
}

// The region's entry ranges [rec begin, rec end, source begin, source end) (FP32
// flow with receivers or extra sources; zeros otherwise).
static __device__ __noinline__ void flow_region_ranges(const FlowArgs &f, int rem, int *out) {
    out[0] = out[1] = out[2] = out[3] = 0;
    if (f.rec_start) {
        out[0] = f.rec_start[rem];
        out[1] = f.rec_start[rem + 1];
    }
    if (f.xs_start) {
        out[2] = f.xs_start[rem];
        out[3] = f.xs_start[rem + 1];
    }
}

// EX: the FP32 variant with receivers and extra sources handled per item; the
// plain variant carries none of that code.
template <int R, int FORM, int LZ, int W, int YB = 1, typename T = float, bool EX = false>
__global__ void __launch_bounds__(32 * W, (tma_warps_per_sm(R, YB) / W > 0 ? tma_warps_per_sm(R, YB) / W : 1))
    fd_tma_flow_kernel(const __grid_constant__ FlowArgs f, int check) {
    static_assert(std::is_same<T, float>::value || std::is_same<T, __nv_bfloat16>::value,
                  "the flow schedule stores FP32 or BF16 (FP16 needs per-level scales)");
    static_assert(!EX || std::is_same<T, float>::value, "receivers and extra sources ride on the FP32 flow only");
    extern __shared__ __align__(128) unsigned char smem_dyn[];
    // item slots: the item of iteration i sits in s_item[i & 1]; thread 0 claims the
    // next one while the current one runs (claims stay in increasing order per CTA,
    // so the lowest unfinished item is always being worked on)
    __shared__ int s_item[2];
    __shared__ int s_fail;
    __shared__ int s_ranges[4];  // the item's receiver and extra-source entries (EX)
    unsigned char *ring = tma_ring_init<R>(smem_dyn);
    const ScaleState sc0 = flow_scales<T>(f, true), sc1 = flow_scales<T>(f, false);
    const int per_plane = f.nbz * f.nby;
    const int per_step = per_plane * f.nbx;
    const int total = per_step * f.nt;
    if (threadIdx.x == 0) s_item[0] = atomicAdd(f.counter, 1);
    int g = 0;
    TmaAcc acc;
    bool ok_all = true;
    for (int iter = 0;; ++iter) {
        __syncthreads();  // s_item[iter & 1] is set; every thread is done with the previous item
        const int item = s_item[iter & 1];
        if (item >= total) break;
        if (threadIdx.x == 0) s_item[(iter + 1) & 1] = atomicAdd(f.counter, 1);
        const int s = item / per_step, rem = item - s * per_step;
        const int bx = rem / per_plane, r2 = rem - bx * per_plane;
        const int by = r2 / f.nbz, bz = r2 - by * f.nbz;
        const int p = (f.cur0 + s) & 1;
        const StepArgs &a = f.a[p];  // parameter space
        if (threadIdx.x < 32) {
            // lane l < 27 checks neighbour (l / 9 - 1, (l / 3) % 3 - 1, l % 3 - 1) of step s - 1
            bool ok = true;
            const int l = threadIdx.x;
            if (s > 0 && l < 27) {
                const int nx = bx + l / 9 - 1, ny = by + (l / 3) % 3 - 1, nz = bz + l % 3 - 1;
                if (nx >= 0 && nx < f.nbx && ny >= 0 && ny < f.nby && nz >= 0 && nz < f.nbz)
                    ok = flow_wait(&f.flags[nx * per_plane + ny * f.nbz + nz], unsigned(s), f.abort);
            }
            if constexpr (EX) {
                // lane 31 waits on no neighbour: it fetches the item's entry ranges meanwhile
                if (l == 31) flow_region_ranges(f, rem, s_ranges);
            }
            ok = __all_sync(0xffffffffu, ok);
            if (l == 0) {
                // the copy engine reads what the acquired flags published
                if (s > 0) asm volatile("fence.proxy.async.global;" ::: "memory");
                s_fail = ok ? 0 : 1;
            }
        }
        __syncthreads();
        if (s_fail) {
            ok_all = false;
            break;
        }
        if constexpr (EX) {
            if (s_ranges[1] > s_ranges[0]) flow_sample_receivers(f, a, s, s_ranges[0], s_ranges[1]);
        }
        const int xb = bx * a.x_block;
        if (!tma_segment<R, FORM, LZ, W, T, kModeStep, true, YB>(&f.maps[p], a, s == 0 ? sc0 : sc1, bz, by, xb,
                                                                 min(xb + a.x_block, a.Nx), ring, g, acc, nullptr,
                                                                 f.step0 + s)) {
            ok_all = false;  // a ring wait gave up (status set); the ring's phases are no longer known
            break;
        }
        __syncthreads();  // the item's stores precede the flag
        if constexpr (EX) {
            if (s_ranges[3] > s_ranges[2]) {
                flow_inject_extra(f, a, s, s_ranges[2], s_ranges[3], FORM == kExpanded);
                __syncthreads();  // and the added sources
            }
        }
        if (threadIdx.x == 0) {
            __threadfence();
            st_release_u32(&f.flags[rem], unsigned(s + 1));
        }
    }
    if (!ok_all) {
        if (threadIdx.x == 0) {
            if (f.a[0].status) atomicOr(f.a[0].status, kStatusTimeout);
            atomicExch(f.abort, 1u);  // the other CTAs stop waiting and leave
        }
        return;
    }
    if constexpr (Io<T>::kScaled) {
        // maxima of the stored (unscaled) values of every level written, the range check
        tma_finish<T>(acc, sc1);
        unsigned bits = acc.amax_bits, dbits = acc.damax_bits;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            bits = max(bits, __shfl_xor_sync(0xffffffffu, bits, o));
            dbits = max(dbits, __shfl_xor_sync(0xffffffffu, dbits, o));
        }
        const unsigned any_over = __any_sync(0xffffffffu, acc.over);
        if ((threadIdx.x & 31) == 0) {
            atomicMax(&f.amax[0], bits);
            atomicMax(&f.amax[1], dbits);
            if (f.a[0].status && (bits >= 0x7f800000u || dbits >= 0x7f800000u || any_over))
                atomicOr(f.a[0].status, kStatusNonFinite);
        }
    } else {
        if (check) reduce_amax(f.a[0], acc.amax_bits, acc.over, acc.damax_bits);
    }
}

template <int R, int FORM, int LZ, int W, int YB = 1, typename T = float, bool EX = false>
cudaError_t tma_flow_launch(const FlowArgs &f, int ctas, bool check, cudaStream_t s) {
    using G = TmaShape<R, LZ, W, T, 0, YB>;
    auto kernel = fd_tma_flow_kernel<R, FORM, LZ, W, YB, T, EX>;
    static bool attr_set = false;
    if (!attr_set) {
        cudaError_t e = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, G::SMEM_BYTES);
        if (e != cudaSuccess) return e;
        attr_set = true;
    }
    kernel<<<ctas, 32 * W, G::SMEM_BYTES, s>>>(f, check ? 1 : 0);
    return cudaGetLastError();
}

template <int R, int FORM, int LZ, int W, int YB = 1, typename T = float, bool EX = false>
int tma_flow_occupancy() {
    using G = TmaShape<R, LZ, W, T, 0, YB>;
    auto kernel = fd_tma_flow_kernel<R, FORM, LZ, W, YB, T, EX>;
    if (cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, G::SMEM_BYTES) != cudaSuccess)
        return 0;
    int n = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, kernel, 32 * W, G::SMEM_BYTES) != cudaSuccess) return 0;
    return n;
}

template <int R>
cudaError_t tma_flow_r(int form, int storage, int tile_z, int tile_y, int rows, bool ex, const FlowArgs &f,
                       int ctas, bool check, cudaStream_t s) {
#define FDGB_FLOW_CASE(LZ, W, YB)                                                                        \
    if (tile_z == 4 * (LZ) && tile_y == YB * (32 / (LZ)) * (W) && rows == YB && storage == kF32) {       \
        if (ex)                                                                                          \
            return form == kFactored ? tma_flow_launch<R, kFactored, LZ, W, YB, float, true>(f, ctas, check, s) \
                                     : tma_flow_launch<R, kExpanded, LZ, W, YB, float, true>(f, ctas, check, s); \
        return form == kFactored ? tma_flow_launch<R, kFactored, LZ, W, YB>(f, ctas, check, s)           \
                                 : tma_flow_launch<R, kExpanded, LZ, W, YB>(f, ctas, check, s);          \
    }
#define FDGB_FLOW_CASE16(LZ, W, YB)                                                             \
    if (tile_z == 4 * (LZ) && tile_y == YB * (32 / (LZ)) * (W) && rows == YB && storage == kBF16 && \
        form == kFactored && !ex)                                                               \
        return tma_flow_launch<R, kFactored, LZ, W, YB, __nv_bfloat16>(f, ctas, check, s);
#define FDGB_FLOW_1(LZ, W) FDGB_FLOW_CASE(LZ, W, 1)
#define FDGB_FLOW_2(LZ, W) FDGB_FLOW_CASE(LZ, W, 2) FDGB_FLOW_CASE16(LZ, W, 2)
#define FDGB_FLOW_16(LZ, W) FDGB_FLOW_CASE16(LZ, W, 1)
    if constexpr (R <= 8) {
        FDGB_TMA_CONFIGS(FDGB_FLOW_1)
        FDGB_TMA_CONFIGS_16(FDGB_FLOW_16)
        FDGB_TMA_CONFIGS2(FDGB_FLOW_2)
    } else {
        FDGB_TMA_CONFIGS_HIGH(FDGB_FLOW_1)
        FDGB_TMA_CONFIGS_16_HIGH(FDGB_FLOW_16)
    }
#undef FDGB_FLOW_1
#undef FDGB_FLOW_2
#undef FDGB_FLOW_16
#undef FDGB_FLOW_CASE
#undef FDGB_FLOW_CASE16
    return cudaErrorInvalidValue;
}

template <int R>
int tma_flow_occ_r(int form, int storage, int tile_z, int tile_y, int rows, bool ex) {
#define FDGB_FLOW_OCC(LZ, W, YB)                                                                \
    if (tile_z == 4 * (LZ) && tile_y == YB * (32 / (LZ)) * (W) && rows == YB && storage == kF32) { \
        if (ex)                                                                                 \
            return form == kFactored ? tma_flow_occupancy<R, kFactored, LZ, W, YB, float, true>() \
                                     : tma_flow_occupancy<R, kExpanded, LZ, W, YB, float, true>(); \
        return form == kFactored ? tma_flow_occupancy<R, kFactored, LZ, W, YB>()                \
                                 : tma_flow_occupancy<R, kExpanded, LZ, W, YB>();               \
    }
#define FDGB_FLOW_OCC16(LZ, W, YB)                                                              \
    if (tile_z == 4 * (LZ) && tile_y == YB * (32 / (LZ)) * (W) && rows == YB && storage == kBF16 && \
        form == kFactored && !ex)                                                               \
        return tma_flow_occupancy<R, kFactored, LZ, W, YB, __nv_bfloat16>();
#define FDGB_FLOW_1(LZ, W) FDGB_FLOW_OCC(LZ, W, 1)
#define FDGB_FLOW_2(LZ, W) FDGB_FLOW_OCC(LZ, W, 2) FDGB_FLOW_OCC16(LZ, W, 2)
#define FDGB_FLOW_16(LZ, W) FDGB_FLOW_OCC16(LZ, W, 1)
    if constexpr (R <= 8) {
        FDGB_TMA_CONFIGS(FDGB_FLOW_1)
        FDGB_TMA_CONFIGS_16(FDGB_FLOW_16)
        FDGB_TMA_CONFIGS2(FDGB_FLOW_2)
    } else {
        FDGB_TMA_CONFIGS_HIGH(FDGB_FLOW_1)
        FDGB_TMA_CONFIGS_16_HIGH(FDGB_FLOW_16)
    }
#undef FDGB_FLOW_1
#undef FDGB_FLOW_2
#undef FDGB_FLOW_16
#undef FDGB_FLOW_OCC
#undef FDGB_FLOW_OCC16
    return 0;
}

// Batch flow (FP32): one persistent launch advances every shot of a batch by nt
// steps. Resident CTAs claim (step, work-list entry) items step-major; each item
// runs the single-shot segment code on its shot's step arguments, which warp 1
// copies into shared memory while warp 0 checks the dependencies (the 27 items
// of step s - 1 around it in its own shot) and thread 0, which issues the bulk
// copies, acquires the shot's tensor maps (once per shot and launch). Every
// dependency has a lower item number, so the waits end (and are bounded all the
// same). Each item reduces its non-finite check into its own shot's status word.
template <int R, int FORM, int LZ, int W>
__global__ void __launch_bounds__(32 * W, (tma_warps_per_sm(R) / W > 0 ? tma_warps_per_sm(R) / W : 1))
    fd_tma_batch_flow_kernel(const __grid_constant__ BatchFlowArgs f) {
    static_assert(W >= 2, "warp 1 copies the arguments");
    static_assert(sizeof(StepArgs) % 8 == 0, "arguments copied 8 bytes per lane");
    extern __shared__ __align__(128) unsigned char smem_dyn[];
    __shared__ __align__(16) StepArgs sa;
    __shared__ const TmaMaps *s_maps;
    __shared__ long long s_step;
    __shared__ int s_item[2];
    __shared__ int s_fail;
    // (shot, parity) pairs whose maps thread 0 has acquired for the copy engine in this
    // launch (the maps do not change during a launch): one bit each, the first shots
    constexpr int kFenceWords = 16;
    __shared__ unsigned s_fenced[kFenceWords];
    if (threadIdx.x < kFenceWords) s_fenced[threadIdx.x] = 0u;
    unsigned char *ring = tma_ring_init<R>(smem_dyn);  // (its barrier orders the zeroing)
    const ScaleState sc{1.0f, 1.0f, 1.0f, 1.0f, 1.0f, 1.0f, 1.0f};
    const int total = f.n_items * f.nt;
    if (threadIdx.x == 0) s_item[0] = atomicAdd(f.counter, 1);
    int g = 0;
    bool ok_all = true;
    for (int iter = 0;; ++iter) {
        __syncthreads();  // s_item[iter & 1] is set; every thread is done with the previous item
        const int item = s_item[iter & 1];
        if (item >= total) break;
        const int s = item / f.n_items, w = item - s * f.n_items;
        const int4 it = __ldg(f.items + w);  // (shot, bz, by, bx)
        if (threadIdx.x < 32) {
            const int l = threadIdx.x;
            if (l == 0) s_item[(iter + 1) & 1] = atomicAdd(f.counter, 1);
            bool ok = true;
            if (s > 0 && l < 27) {
                const int4 ge = __ldg(f.geo + it.x);  // z tiles, y tiles, x-chunks, first entry
                const int nx = it.w + l / 9 - 1, ny = it.z + (l / 3) % 3 - 1, nz = it.y + l % 3 - 1;
                if (nx >= 0 && nx < ge.z && ny >= 0 && ny < ge.y && nz >= 0 && nz < ge.x)
                    ok = flow_wait(&f.flags[ge.w + (nx * ge.y + ny) * ge.x + nz], unsigned(s), f.abort);
            }
            ok = __all_sync(0xffffffffu, ok);
            if (l == 0) {
                // the copy engine reads what the acquired flags published
                if (s > 0) asm volatile("fence.proxy.async.global;" ::: "memory");
                s_fail = ok ? 0 : 1;
                // the maps were written to global memory by the host: thread 0, which issues
                // the copies, acquires them for the copy engine once per launch
                const BatchShot *sh = f.shots + it.x;
                const int p = (__ldg(&sh->cur0) + s) & 1;
                const int bit = 2 * it.x + p;
                const bool known = bit < 32 * kFenceWords && ((s_fenced[bit >> 5] >> (bit & 31)) & 1u);
                if (!known) {
                    const CUtensorMap *m[5] = {&sh->maps[p].u_halo, &sh->maps[p].u_pt, &sh->maps[p].up_pt,
                                               &sh->maps[p].f1_pt, &sh->maps[p].f2_pt};
#pragma unroll
                    for (int k = 0; k < 5; ++k)
                        asm volatile("fence.proxy.tensormap::generic.acquire.gpu [%0], 128;" ::"l"(
                                         reinterpret_cast<uint64_t>(m[k]))
                                     : "memory");
                    if (bit < 32 * kFenceWords) s_fenced[bit >> 5] |= 1u << (bit & 31);
                }
            }
        } else if (threadIdx.x < 64) {
            const int l = threadIdx.x - 32;
            const BatchShot *sh = f.shots + it.x;
            const int p = (__ldg(&sh->cur0) + s) & 1;
            constexpr int n8 = int(sizeof(StepArgs) / 8);
            const long long *src = reinterpret_cast<const long long *>(&sh->args[p]);
            long long *dst = reinterpret_cast<long long *>(&sa);
            for (int i = l; i < n8; i += 32) dst[i] = __ldg(src + i);
            __syncwarp();
            if (l == 0) {
                s_step = __ldg(&sh->step0) + s;
                sa.step = s_step;
                s_maps = &sh->maps[p];
            }
        }
        __syncthreads();
        if (s_fail) {
            ok_all = false;
            break;
        }
        const int xb = it.w * sa.x_block;
        TmaAcc acc;
        if (!tma_segment<R, FORM, LZ, W, float, kModeStep, true>(s_maps, sa, sc, it.y, it.z, xb,
                                                                 min(xb + sa.x_block, sa.Nx), ring, g, acc, nullptr,
                                                                 s_step)) {
            ok_all = false;  // a ring wait gave up (status set); the ring's phases are no longer known
            break;
        }
        reduce_amax(sa, acc.amax_bits, acc.over, acc.damax_bits);
        __syncthreads();  // the item's stores precede the flag; every thread is done with sa
        if (threadIdx.x == 0) {
            __threadfence();
            st_release_u32(&f.flags[w], unsigned(s + 1));
        }
    }
    if (!ok_all && threadIdx.x == 0) {
        if (sa.status) atomicOr(sa.status, kStatusTimeout);
        atomicExch(f.abort, 1u);  // the other CTAs stop waiting and leave
    }
}

template <int R, int FORM, int LZ, int W>
cudaError_t tma_batch_flow_launch(const BatchFlowArgs &f, int ctas, cudaStream_t s) {
    using G = TmaShape<R, LZ, W, float>;
    auto kernel = fd_tma_batch_flow_kernel<R, FORM, LZ, W>;
    static bool attr_set = false;
    if (!attr_set) {
        cudaError_t e = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, G::SMEM_BYTES);
        if (e != cudaSuccess) return e;
        attr_set = true;
    }
    kernel<<<ctas, 32 * W, G::SMEM_BYTES, s>>>(f);
    return cudaGetLastError();
}

template <int R, int FORM, int LZ, int W>
int tma_batch_flow_occupancy() {
    using G = TmaShape<R, LZ, W, float>;
    auto kernel = fd_tma_batch_flow_kernel<R, FORM, LZ, W>;
    if (cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, G::SMEM_BYTES) != cudaSuccess)
        return 0;
    int n = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, kernel, 32 * W, G::SMEM_BYTES) != cudaSuccess) return 0;
    return n;
}

// The batch tiles: 32x16 (LZ 8, W 4) and 64x8 (LZ 16, W 4).
template <int R>
cudaError_t tma_batch_flow_r(int form, int tile_z, int tile_y, const BatchFlowArgs &f, int ctas, cudaStream_t s) {
    if constexpr (R > kMaxBatchRadius) {
        return cudaErrorInvalidValue;
    } else {
#define FDGB_BFLOW_CASE(LZ, W)                                                                   \
    if (tile_z == 4 * (LZ) && tile_y == (32 / (LZ)) * (W))                                       \
        return form == kFactored ? tma_batch_flow_launch<R, kFactored, LZ, W>(f, ctas, s)         \
                                 : tma_batch_flow_launch<R, kExpanded, LZ, W>(f, ctas, s);
        FDGB_BFLOW_CASE(8, 4)
        FDGB_BFLOW_CASE(16, 4)
#undef FDGB_BFLOW_CASE
        return cudaErrorInvalidValue;
    }
}

template <int R>
int tma_batch_flow_occ_r(int form, int tile_z, int tile_y) {
    if constexpr (R > kMaxBatchRadius) {
        return 0;
    } else {
#define FDGB_BFLOW_OCC(LZ, W)                                                                    \
    if (tile_z == 4 * (LZ) && tile_y == (32 / (LZ)) * (W))                                       \
        return form == kFactored ? tma_batch_flow_occupancy<R, kFactored, LZ, W>()                \
                                 : tma_batch_flow_occupancy<R, kExpanded, LZ, W>();
        FDGB_BFLOW_OCC(8, 4)
        FDGB_BFLOW_OCC(16, 4)
#undef FDGB_BFLOW_OCC
        return 0;
    }
}

}  // namespace fdgb

#define FDGB_INSTANTIATE_FLOW_RADIUS(R)                                                           \
    namespace fdgb {                                                                              \
    cudaError_t tma_flow_radius_##R(int form, int storage, int tile_z, int tile_y, int rows, bool ex, \
                                    const FlowArgs &f, int ctas, bool check, cudaStream_t s) {    \
        return tma_flow_r<R>(form, storage, tile_z, tile_y, rows, ex, f, ctas, check, s);         \
    }                                                                                             \
    int tma_flow_occ_radius_##R(int form, int storage, int tile_z, int tile_y, int rows, bool ex) { \
        return tma_flow_occ_r<R>(form, storage, tile_z, tile_y, rows, ex);                        \
    }                                                                                             \
    cudaError_t tma_batch_flow_radius_##R(int form, int tile_z, int tile_y, const BatchFlowArgs &f, \
                                          int ctas, cudaStream_t s) {                             \
        return tma_batch_flow_r<R>(form, tile_z, tile_y, f, ctas, s);                             \
    }                                                                                             \
    int tma_batch_flow_occ_radius_##R(int form, int tile_z, int tile_y) {                         \
        return tma_batch_flow_occ_r<R>(form, tile_z, tile_y);                                     \
    }                                                                                             \
    }
