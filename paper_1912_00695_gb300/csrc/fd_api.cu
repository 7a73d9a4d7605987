// C-ABI of the single-shot solver (include/fd_acoustic.h): handle lifetime,
// model upload and validation, sources, graph-replayed time stepping, the
// launch-shape autotuner and read-back.
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <algorithm>
#include <cstdlib>
#include <map>
#include <mutex>
#include <string>
#include <tuple>
#include <vector>

#include "../../include/fd_acoustic.h"
#include "fd_internal.h"
#include "fd_flow.h"
#include "fd_launch_count.h"
#include "fd_periodic.h"

using namespace fdgb;

namespace {

thread_local std::string g_last_error;

int fail(int code, const char *fmt, ...) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    std::vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    g_last_error = buf;
    return code;
}

#define FD_CUDA(expr)                                                                      \
    do {                                                                                   \
        cudaError_t e_ = (expr);                                                           \
        if (e_ != cudaSuccess)                                                             \
            return fail(FD_ECUDA, "%s failed: %s", #expr, cudaGetErrorString(e_));         \
    } while (0)

size_t elem_size(int storage) { return storage == kF32 ? 4 : 2; }

struct Source {
    int x, y, z;  // computational-domain node
    std::vector<float> wavelet;
};

struct GraphEntry {
    cudaGraphExec_t exec = nullptr;
    int nt = 0, cur = 0;
    long long launches = 0;  // kernel launches one replay executes
    bool flow = false;       // the flow schedule (one persistent launch for the nt steps)
    long long step0 = 0;
    unsigned long long gen = 0;
};

// Process-wide launch-shape cache:
// (Nx, Ny, Nz, radius, storage, form, check, kernel) -> (tile_z, tile_y, x_block)
std::mutex g_tune_mu;
std::map<std::tuple<int, int, int, int, int, int, int, int>, std::tuple<int, int, int, int>> g_tune_cache;
// two-step kernel: (Nx, Ny, Nz, radius) -> x_block
std::map<std::tuple<int, int, int, int>, int> g_tb_cache;
// flow schedule: (Nx, Ny, Nz, radius, form, tile_z, tile_y) -> (x_block, faster than per-step launches)
std::map<std::tuple<int, int, int, int, int, int, int, int>, std::pair<int, bool>> g_flow_cache;

// Device memory is stream-ordered (cudaMallocAsync / cudaFreeAsync) from the
// device's default pool, whose release threshold is raised once per device so
// that freed blocks stay cached: shots created and retired at a high rate (a
// serving loop) reuse memory without driver allocations, and freeing a shot's
// fields never synchronises the device (a plain cudaFree would stall every
// stream, including other batches' launches).
std::mutex g_pool_mu;
bool g_pool_ready[64] = {};

cudaError_t dev_alloc(void **p, size_t bytes, cudaStream_t s) {
    *p = nullptr;
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev >= 0 && dev < 64) {
        std::lock_guard<std::mutex> lk(g_pool_mu);
        if (!g_pool_ready[dev]) {
            cudaMemPool_t pool;
            if (cudaDeviceGetDefaultMemPool(&pool, dev) == cudaSuccess) {
                cuuint64_t thr = ~cuuint64_t(0);
                cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &thr);
            }
            cudaGetLastError();
            g_pool_ready[dev] = true;
        }
    }
    e = cudaMallocAsync(p, bytes, s);
    if (e != cudaSuccess) {
        *p = nullptr;
        return e;
    }
    if (reinterpret_cast<uintptr_t>(*p) % 256 != 0) {  // the bulk tensor copies need aligned bases
        cudaFreeAsync(*p, s);
        *p = nullptr;
        return cudaErrorMisalignedAddress;
    }
    return cudaSuccess;
}

void dev_free(void *p, cudaStream_t s) {
    if (p) cudaFreeAsync(p, s);
}

using EncodeTiledFn = CUresult (*)(CUtensorMap *, CUtensorMapDataType, cuuint32_t, void *,
                                   const cuuint64_t *, const cuuint64_t *, const cuuint32_t *,
                                   const cuuint32_t *, CUtensorMapInterleave, CUtensorMapSwizzle,
                                   CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

// cuTensorMapEncodeTiled through the runtime's driver entry-point lookup (no
// link-time dependency on the driver library).
EncodeTiledFn encode_fn() {
    static EncodeTiledFn fn = nullptr;
    static std::once_flag once;
    std::call_once(once, [] {
        void *p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<EncodeTiledFn>(p);
    });
    return fn;
}

// Launch shapes of the TMA kernel: tile (z, y) and y rows per thread.
struct TileShape {
    int tz, ty, rows;
};

// The TMA kernel's shapes for a storage/form.
std::vector<TileShape> tma_tiles(int storage, int form, int radius) {
    if (radius > 8) {  // space orders 18-24: 32-wide tiles only, one row per thread
        if (storage == kF32) return {{32, 32, 1}, {32, 16, 1}};
        if (form == kFactored) return {{32, 16, 1}};
        return {};
    }
    if (storage == kF32)
        return {{32, 32, 1}, {64, 16, 1}, {128, 8, 1}, {32, 16, 1}, {64, 8, 1}, {32, 32, 2}, {64, 16, 2}};
    if (form == kFactored) return {{32, 16, 1}, {64, 8, 1}, {32, 32, 2}, {64, 16, 2}};
    return {};
}

bool shape_matches(const TileShape &p, int tz, int ty, int rows) {
    return (tz == 0 || tz == p.tz) && (ty == 0 || ty == p.ty) && (rows == 0 || rows == p.rows);
}

// Valid (tile_z, tile_y, rows) requests of each kernel (0 = any).
bool tile_ok(int kernel, int storage, int form, int radius, int tz, int ty, int rows) {
    if (kernel == kStream)
        return (tz == 0 || tz == 32) && (ty == 0 || ty == 4 || ty == 8 || ty == 16) && rows <= 1;
    if (kernel == kTma) {
        for (auto &p : tma_tiles(storage, form, radius))
            if (shape_matches(p, tz, ty, rows)) return true;
        return false;
    }
    return rows <= 1;
}

}  // namespace

namespace fdgb {
void set_last_error(const char *msg) { g_last_error = msg; }
}  // namespace fdgb

struct fd_handle {
    int nx = 0, ny = 0, nz = 0, nbl = 0, k = 0, r = 0;
    double h = 0, dt = 0;
    int Nx = 0, Ny = 0, Nz = 0, pz = 0;
    long long plane = 0;
    size_t n_pitched = 0;
    fd_options opt{};
    int tile_z = 0, tile_y = 0, x_block = 0, kernel = kStream;
    int rows = 1;  // y rows per thread of the TMA kernel
    TmaMaps tmaps[2];  // TMA kernel: maps of the step whose u^n is ubuf[0] / ubuf[1]
    void *ubuf[2] = {nullptr, nullptr};
    void *dbuf = nullptr;  // 16-bit storage: the increment d^n = u^n - u^{n-1}
    float *f1 = nullptr, *f2 = nullptr;
    float *d_wavelet = nullptr;
    int *d_src = nullptr;  // 3 * ns ints: x[], y[], z[]
    int ld = 0;
    std::vector<Source> sources;
    unsigned *d_status = nullptr;
    LevelScales *d_scales = nullptr;
    ModelCheck *d_check = nullptr;
    float *d_unpack = nullptr;
    long long step = 0;
    int cur = 0;  // ubuf[cur] holds u^step
    cudaStream_t own_stream = nullptr, stream = nullptr;
    bool has_model = false;
    int box[6] = {0, 0, 0, 0, 0, 0};
    float src_bound = 0.0f;
    double coef_c[kMaxRadius + 1] = {};
    std::vector<GraphEntry> graphs;
    unsigned long long gen = 1;
    cudaEvent_t ev0 = nullptr, ev1 = nullptr;
    bool timed = false;
    bool extra_distinct = true;  // sources beyond the fused ones sit at pairwise distinct nodes
    // two-step kernel: the pair of output buffers, its x_block and tensor maps by input pair
    void *tb_buf[2] = {nullptr, nullptr};
    int tb_xb = 0;
    // flow schedule: work counter, abort word and per-item flags; resident CTAs of its kernel
    void *flow_buf = nullptr;
    size_t flow_bytes = 0;
    int flow_ctas = 0, flow_ctas_ex = 0;  // resident CTAs: plain flow kernel / receivers + extra sources variant
    int flow_xb = 0;         // the flow schedule's x_block, timed, cached or forced (0: not yet)
    int flow_run_xb = 0;     // the x_block the flow graphs are recorded with
    bool flow_wins = true;   // the flow beat per-step launches when the two were timed
    int flow_extras = -1;    // receivers (1) / extra sources (2) present when flow_xb was chosen
    struct TbMaps {
        const void *u, *up;
        TmaMaps maps;
    };
    std::vector<TbMaps> tb_maps;
    // slab of a shot split along x (fd_slab_create): the buffers hold planes
    // [x_off, x_off + Nx) of a domain of Nx_glob planes; the step updates local planes
    // [x_lo, x_hi) and reads ghost_lo / ghost_hi planes of the neighbours' data below
    // and above them. An ordinary handle is its own single slab.
    bool slab = false;
    int device = 0;  // the CUDA device the buffers live on (current at creation)
    int x_off = 0, Nx_glob = 0, x_lo = 0, x_hi = 0, ghost_lo = 0, ghost_hi = 0;
    // receivers: 8 (pitched offset, weight) pairs each; traces [n_rec][rec_nt_max]
    int n_rec = 0, rec_nt_max = 0;
    long long rec_step0 = 0;
    long long *d_rec_off = nullptr;
    float *d_rec_w = nullptr;
    float *d_traces = nullptr;
    std::vector<int> rec_node;  // lower corner node (x, y, z) of each receiver
    std::vector<long long> rec_off_h;  // host copies of the receivers' corner offsets and weights
    std::vector<float> rec_w_h;
    // flow schedule with receivers or extra sources (FP32): the per-region entry
    // tables, built for one x_block and the handle's state (gen)
    unsigned char *d_flow_tab = nullptr;
    size_t flow_tab_bytes = 0;
    unsigned long long flow_tab_gen = 0;
    int flow_tab_xb = 0;
};

// (defined with the forward path, with C linkage)
extern "C" {
static bool flow_eligible(const fd_handle *hd);
}

namespace {

bool check_enabled(const fd_handle *hd) { return hd->opt.check_finite != 0 || hd->opt.storage != kF32; }

StepArgs make_args(const fd_handle *hd, long long step, int cur) {
    StepArgs a{};
    a.u = hd->ubuf[cur];
    if (hd->opt.storage == kF32) {
        a.up = hd->ubuf[cur ^ 1];
        a.un = nullptr;
    } else {
        a.up = hd->dbuf;
        a.un = hd->ubuf[cur ^ 1];
    }
    a.f1 = hd->f1;
    a.f2 = hd->f2;
    a.Nx = hd->Nx;
    a.Ny = hd->Ny;
    a.Nz = hd->Nz;
    a.pz = hd->pz;
    a.plane = hd->plane;
    a.x_block = hd->x_block > 0 ? hd->x_block : hd->Nx;
    a.x_lo = hd->x_lo;
    a.x_hi = hd->x_hi;
    a.bx0 = hd->box[0];
    a.bx1 = hd->box[1];
    a.by0 = hd->box[2];
    a.by1 = hd->box[3];
    a.bz0 = hd->box[4];
    a.bz1 = hd->box[5];
    const double inv_h2 = 1.0 / (hd->h * hd->h);
    const double scale = hd->opt.form == kExpanded ? hd->dt * hd->dt * inv_h2 : inv_h2;
    for (int j = 0; j <= kMaxRadius; ++j) a.coef[j] = 0.0f;
    a.coef[0] = float(3.0 * hd->coef_c[0] * scale);
    for (int j = 1; j <= hd->r; ++j) a.coef[j] = float(hd->coef_c[j] * scale);
    a.half_dt = float(0.5 * hd->dt);
    a.dt2 = float(hd->dt * hd->dt);
    const int ns = int(hd->sources.size());
    a.ns = ns < kFusedSources ? ns : kFusedSources;
    for (int s = 0; s < a.ns; ++s) {
        a.sx[s] = hd->sources[s].x;
        a.sy[s] = hd->sources[s].y;
        a.sz[s] = hd->sources[s].z;
    }
    a.wavelet = hd->d_wavelet;
    a.ld = hd->ld;
    a.step = step;
    a.status = check_enabled(hd) ? hd->d_status : nullptr;
    a.scales = hd->opt.storage != kF32 ? hd->d_scales : nullptr;
    a.src_bound = hd->src_bound;
    // receivers: the TMA kernel samples its input level u^step (sample step - s0 - 1)
    a.rec_off = hd->d_rec_off;
    a.rec_w = hd->d_rec_w;
    a.traces = hd->d_traces;
    a.n_rec = hd->kernel == kTma ? hd->n_rec : 0;
    a.rec_stride = hd->rec_nt_max;
    const long long smp = step - hd->rec_step0 - 1;
    a.rec_sample = (a.n_rec > 0 && smp >= 0 && smp < hd->rec_nt_max) ? int(smp) : -1;
    return a;
}

// Standalone sample of level `level` (stored in buffer u) into the traces.
cudaError_t sample_level(const fd_handle *hd, const void *u, long long level, cudaStream_t s) {
    const long long smp = level - hd->rec_step0 - 1;
    if (hd->n_rec <= 0 || smp < 0 || smp >= hd->rec_nt_max) return cudaSuccess;
    return launch_sample_receivers(u, hd->opt.storage, hd->d_scales, int((level % 3 + 3) % 3), hd->d_rec_off,
                                   hd->d_rec_w, hd->n_rec, hd->d_traces + smp, hd->rec_nt_max, s);
}

// One step with the given launch shape; `map` holds the tensor maps of this step
// (TMA kernel only).
cudaError_t launch_kernel(const fd_handle *hd, const StepArgs &a, int kernel, int tile_z, int tile_y, int rows,
                          const TmaMaps *map, bool check, cudaStream_t s) {
    if (hd->opt.boundary == FD_BOUNDARY_PERIODIC) return launch_periodic_step(hd->r, hd->opt.form, a, check, s);
    if (kernel == kNaive) return launch_naive_step(hd->r, hd->opt.form, hd->opt.storage, a, check, s);
    if (kernel == kTma)
        return launch_tma_step(hd->r, hd->opt.form, hd->opt.storage, tile_z, tile_y, rows, *map, a, check, s);
    return launch_stream_step(hd->r, hd->opt.form, hd->opt.storage, tile_y, a, check, s);
}

cudaError_t enqueue_step(const fd_handle *hd, const StepArgs &a, cudaStream_t s) {
    const bool check = check_enabled(hd);
    const TmaMaps *map = a.u == hd->ubuf[0] ? &hd->tmaps[0] : &hd->tmaps[1];
    cudaError_t e = launch_kernel(hd, a, hd->kernel, hd->tile_z, hd->tile_y, hd->rows, map, check, s);
    if (e != cudaSuccess) return e;
    const int ns = int(hd->sources.size());
    if (ns > kFusedSources)
        e = launch_inject_extra(a, hd->d_src, hd->d_src + ns, hd->d_src + 2 * ns, kFusedSources,
                                ns - kFusedSources, hd->opt.storage, hd->opt.form == kExpanded,
                                hd->extra_distinct, s);
    if (e == cudaSuccess && hd->n_rec > 0 && hd->kernel != kTma)
        // kernels without fused sampling: sample the level this step wrote (FP32: over u^{n-1})
        e = sample_level(hd, a.up, a.step + 1, s);
    return e;
}

void destroy_graphs(fd_handle *hd) {
    for (auto &g : hd->graphs)
        if (g.exec) cudaGraphExecDestroy(g.exec);
    hd->graphs.clear();
}

int encode_box(const fd_handle *hd, const void *base, CUtensorMapDataType dtype, int esize, int bw, int bh,
               CUtensorMap *out) {
    EncodeTiledFn fn = encode_fn();
    if (!fn) return fail(FD_ECUDA, "cuTensorMapEncodeTiled is not available from the driver");
    cuuint64_t dims[3] = {cuuint64_t(hd->Nz), cuuint64_t(hd->Ny), cuuint64_t(hd->Nx)};
    cuuint64_t strides[2] = {cuuint64_t(hd->pz) * esize, cuuint64_t(hd->plane) * esize};
    cuuint32_t box[3] = {cuuint32_t(bw), cuuint32_t(bh), 1};
    cuuint32_t estr[3] = {1, 1, 1};
    CUresult r = fn(out, dtype, 3, const_cast<void *>(base), dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                    CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS) return fail(FD_ECUDA, "cuTensorMapEncodeTiled failed (%d)", int(r));
    return FD_OK;
}

// Maps of one step of the TMA kernel with u^n in `u` and u^{n-1} in `up`.
int make_maps(const fd_handle *hd, const void *u, const void *up, int tile_z, int tile_y, int rows, TmaMaps *out) {
    int bw = 0, bh = 0, rz = 0;
    if (!tma_box(hd->r, hd->opt.form, hd->opt.storage, tile_z, tile_y, rows, &bw, &bh, &rz))
        return fail(FD_ENOTSUP, "no TMA tile %dx%d for this storage/form", tile_z, tile_y);
    const int es = int(elem_size(hd->opt.storage));
    const CUtensorMapDataType ut = hd->opt.storage == kF32    ? CU_TENSOR_MAP_DATA_TYPE_FLOAT32
                                   : hd->opt.storage == kBF16 ? CU_TENSOR_MAP_DATA_TYPE_BFLOAT16
                                                              : CU_TENSOR_MAP_DATA_TYPE_FLOAT16;
    int rc = encode_box(hd, u, ut, es, bw, bh, &out->u_halo);
    if (rc == FD_OK) rc = encode_box(hd, u, ut, es, tile_z, tile_y, &out->u_pt);
    if (rc == FD_OK) rc = encode_box(hd, up, ut, es, tile_z, tile_y, &out->up_pt);
    if (rc == FD_OK) rc = encode_box(hd, hd->f1, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 4, tile_z, tile_y, &out->f1_pt);
    if (rc == FD_OK) rc = encode_box(hd, hd->f2, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 4, tile_z, tile_y, &out->f2_pt);
    return rc;
}

int build_maps(fd_handle *hd) {
    if (hd->kernel != kTma) return FD_OK;
    for (int b = 0; b < 2; ++b) {
        const void *up = hd->opt.storage == kF32 ? hd->ubuf[b ^ 1] : hd->dbuf;
        int rc = make_maps(hd, hd->ubuf[b], up, hd->tile_z, hd->tile_y, hd->rows, &hd->tmaps[b]);
        if (rc != FD_OK) return rc;
    }
    return FD_OK;
}

// SMs of the current device (a GB300's 152 if the query fails)
int device_sms() {
    int dev = 0, sms = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || sms <= 0) {
        cudaGetLastError();
        return 152;
    }
    return sms;
}

int heuristic_x_block(const fd_handle *hd, int tile_z, int tile_y) {
    const int tiles = ((hd->Nz + tile_z - 1) / tile_z) * ((hd->Ny + tile_y - 1) / tile_y);
    int chunks = (2 * device_sms() + tiles - 1) / tiles;
    const int max_chunks = hd->Nx / 16 > 0 ? hd->Nx / 16 : 1;
    chunks = std::max(1, std::min(chunks, max_chunks));
    return (hd->Nx + chunks - 1) / chunks;
}

// Pick (tile_z, tile_y, rows, x_block) for the handle's kernel by timing candidate
// launch shapes. The candidates run on scratch wavefields, scale slots and
// status word (zeroed, no sources), so the handle's own state is never touched.
int autotune(fd_handle *hd) {
    const int kernel = hd->kernel;
    const bool force_tile = hd->opt.tile_z > 0 || hd->opt.tile_y > 0 || hd->opt.rows > 0,
               force_xb = hd->opt.x_block > 0;
    std::vector<TileShape> tiles;
    if (kernel == kTma) {
        // a shot that runs the flow schedule by default (FP32, BF16) takes one row per
        // thread unless the options ask for two: two-row shapes time well in single
        // launches but run slower under the flow (fewer resident warps for its items)
        const bool one_row = hd->opt.rows == 0 && hd->opt.kernel == kAuto && flow_eligible(hd);
        for (auto &p : tma_tiles(hd->opt.storage, hd->opt.form, hd->r))
            if (shape_matches(p, hd->opt.tile_z, hd->opt.tile_y, hd->opt.rows) && !(one_row && p.rows > 1))
                tiles.push_back(p);
    } else {
        for (int ty : {4, 8, 16})
            if (hd->opt.tile_y == 0 || hd->opt.tile_y == ty) tiles.push_back({32, ty, 1});
    }
    if (tiles.empty()) return fail(FD_ENOTSUP, "no tile shape matches the options");
    std::vector<int> xbs;
    if (force_xb) {
        xbs.push_back(hd->opt.x_block);
    } else {
        const std::vector<int> cand = kernel == kTma ? std::vector<int>{12, 16, 24, 32, 48, 64, 128}
                                                     : std::vector<int>{16, 32, 64, 128};
        for (int xb : cand)
            if (xb < hd->Nx) xbs.push_back(xb);
        xbs.push_back(hd->Nx);
    }
    // TMA kernel: add the x_block whose CTA count (tiles x chunks) just fits the GPU's
    // resident CTA slots once, twice or three times
    auto tile_xbs = [&](int tz, int ty, int rows) {
        std::vector<int> v = xbs;
        if (kernel != kTma || force_xb) return v;
        int dev = 0, sms = 0;
        if (cudaGetDevice(&dev) != cudaSuccess ||
            cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || sms <= 0) {
            cudaGetLastError();
            return v;
        }
        const long long warps = (long long)tz * ty / (128 * rows);  // 4 points per thread and row
        const long long slots = (long long)sms * std::max(1LL, tma_warps_per_sm(hd->r, rows) / warps);
        const long long tiles = (long long)((hd->Nz + tz - 1) / tz) * ((hd->Ny + ty - 1) / ty);
        for (int waves = 1; waves <= 3; ++waves) {
            const long long chunks = slots * waves / tiles;  // chunks per tile that still fit
            if (chunks < 1) continue;
            const long long xb = (hd->Nx + chunks - 1) / chunks;
            if (xb >= 4 && xb < hd->Nx && std::find(v.begin(), v.end(), int(xb)) == v.end())
                v.push_back(int(xb));
        }
        return v;
    };
    auto take = [&](const TileShape &t, int xb) {
        hd->tile_z = t.tz;
        hd->tile_y = t.ty;
        hd->rows = t.rows;
        hd->x_block = xb;
    };
    if (tiles.size() == 1 && tile_xbs(tiles[0].tz, tiles[0].ty, tiles[0].rows).size() == 1) {
        take(tiles[0], xbs[0]);
        return FD_OK;
    }
    auto key = std::make_tuple(hd->Nx, hd->Ny, hd->Nz, hd->r, hd->opt.storage, hd->opt.form,
                               int(check_enabled(hd)), kernel);
    if (!force_tile && !force_xb) {
        std::lock_guard<std::mutex> lk(g_tune_mu);
        auto it = g_tune_cache.find(key);
        if (it != g_tune_cache.end()) {
            std::tie(hd->tile_z, hd->tile_y, hd->rows, hd->x_block) = it->second;
            return FD_OK;
        }
    }
    const char *env = std::getenv("FDGB_NO_TUNE");
    if (env && env[0] == '1') {
        take(tiles[0], force_xb ? xbs[0] : heuristic_x_block(hd, tiles[0].tz, tiles[0].ty));
        return FD_OK;
    }
    const size_t ub = hd->n_pitched * elem_size(hd->opt.storage);
    const bool inc = hd->opt.storage != kF32;  // increment form needs a third field
    void *s0 = nullptr, *s1 = nullptr, *s2 = nullptr, *aux = nullptr;
    if (dev_alloc(&s0, ub, hd->stream) != cudaSuccess || dev_alloc(&s1, ub, hd->stream) != cudaSuccess ||
        (inc && dev_alloc(&s2, ub, hd->stream) != cudaSuccess) || dev_alloc(&aux, 256, hd->stream) != cudaSuccess) {
        cudaGetLastError();
        dev_free(s0, hd->stream);
        dev_free(s1, hd->stream);
        dev_free(s2, hd->stream);
        dev_free(aux, hd->stream);
        // not enough memory for scratch fields: take the first shape, heuristic x_block
        take(tiles[0], force_xb ? xbs[0] : heuristic_x_block(hd, tiles[0].tz, tiles[0].ty));
        return FD_OK;
    }
    LevelScales *ls = static_cast<LevelScales *>(aux);
    unsigned *st = reinterpret_cast<unsigned *>(static_cast<char *>(aux) + 128);
    int rc = FD_OK;
    float best = 1e30f;
    int best_t = 0, best_xb = xbs[0];
    cudaError_t e = cudaMemsetAsync(s0, 0, ub, hd->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(s1, 0, ub, hd->stream);
    if (e == cudaSuccess && inc) e = cudaMemsetAsync(s2, 0, ub, hd->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(aux, 0, 256, hd->stream);
    if (e == cudaSuccess) e = launch_init_scales(ls, hd->stream);
    StepArgs a = make_args(hd, 0, 0);
    a.u = s0;
    a.up = s1;
    a.un = inc ? s2 : nullptr;
    a.ns = 0;
    a.n_rec = 0;
    a.rec_sample = -1;
    a.scales = hd->opt.storage != kF32 ? ls : nullptr;
    a.status = check_enabled(hd) ? st : nullptr;
    const bool check = check_enabled(hd);
    for (size_t ti = 0; ti < tiles.size() && e == cudaSuccess && rc == FD_OK; ++ti) {
        TmaMaps map;
        const TileShape &t = tiles[ti];
        if (kernel == kTma) rc = make_maps(hd, s0, s1, t.tz, t.ty, t.rows, &map);
        const std::vector<int> xbs = tile_xbs(t.tz, t.ty, t.rows);
        for (size_t xi = 0; xi < xbs.size() && e == cudaSuccess && rc == FD_OK; ++xi) {
            a.x_block = xbs[xi];
            for (int w = 0; w < 2 && e == cudaSuccess; ++w)
                e = launch_kernel(hd, a, kernel, t.tz, t.ty, t.rows, &map, check, hd->stream);
            if (e == cudaSuccess) e = cudaEventRecord(hd->ev0, hd->stream);
            for (int w = 0; w < 4 && e == cudaSuccess; ++w)
                e = launch_kernel(hd, a, kernel, t.tz, t.ty, t.rows, &map, check, hd->stream);
            if (e == cudaSuccess) e = cudaEventRecord(hd->ev1, hd->stream);
            if (e == cudaSuccess) e = cudaEventSynchronize(hd->ev1);
            float ms = 0;
            if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, hd->ev0, hd->ev1);
            if (e == cudaSuccess && ms < best) {
                best = ms;
                best_t = int(ti);
                best_xb = xbs[xi];
            }
        }
    }
    if (e != cudaSuccess && rc == FD_OK) rc = fail(FD_ECUDA, "autotune launch failed: %s", cudaGetErrorString(e));
    dev_free(s0, hd->stream);
    dev_free(s1, hd->stream);
    dev_free(s2, hd->stream);
    dev_free(aux, hd->stream);
    cudaStreamSynchronize(hd->stream);
    if (rc != FD_OK) return rc;
    take(tiles[best_t], best_xb);
    if (!force_tile && !force_xb) {
        std::lock_guard<std::mutex> lk(g_tune_mu);
        g_tune_cache[key] = std::make_tuple(hd->tile_z, hd->tile_y, hd->rows, hd->x_block);
    }
    return FD_OK;
}

int upload_sources(fd_handle *hd) {
    dev_free(hd->d_wavelet, hd->stream);
    dev_free(hd->d_src, hd->stream);
    hd->d_wavelet = nullptr;
    hd->d_src = nullptr;
    const int ns = int(hd->sources.size());
    hd->extra_distinct = true;
    for (int i = kFusedSources; i < ns; ++i)
        for (int j = kFusedSources; j < i; ++j)
            if (hd->sources[i].x == hd->sources[j].x && hd->sources[i].y == hd->sources[j].y &&
                hd->sources[i].z == hd->sources[j].z)
                hd->extra_distinct = false;
    hd->ld = 0;
    for (auto &s : hd->sources) hd->ld = std::max<int>(hd->ld, int(s.wavelet.size()));
    if (ns == 0) return FD_OK;
    std::vector<float> w(size_t(ns) * hd->ld, 0.0f);
    std::vector<int> xyz(3 * size_t(ns));
    for (int s = 0; s < ns; ++s) {
        std::copy(hd->sources[s].wavelet.begin(), hd->sources[s].wavelet.end(),
                  w.begin() + size_t(s) * hd->ld);
        xyz[s] = hd->sources[s].x;
        xyz[ns + s] = hd->sources[s].y;
        xyz[2 * ns + s] = hd->sources[s].z;
    }
    if (dev_alloc(reinterpret_cast<void **>(&hd->d_wavelet), w.size() * sizeof(float), hd->stream) != cudaSuccess ||
        dev_alloc(reinterpret_cast<void **>(&hd->d_src), xyz.size() * sizeof(int), hd->stream) != cudaSuccess)
        return fail(FD_ENOMEM, "cannot allocate source arrays");
    FD_CUDA(cudaMemcpyAsync(hd->d_wavelet, w.data(), w.size() * sizeof(float), cudaMemcpyHostToDevice,
                            hd->stream));
    FD_CUDA(cudaMemcpyAsync(hd->d_src, xyz.data(), xyz.size() * sizeof(int), cudaMemcpyHostToDevice,
                            hd->stream));
    FD_CUDA(cudaStreamSynchronize(hd->stream));
    return FD_OK;
}

// Bound on |dt^2 q / (m + dt/2 eta)| summed over sources, for 16-bit scale selection.
int update_src_bound(fd_handle *hd) {
    double bound = 0.0;
    if (hd->has_model) {
        for (auto &s : hd->sources) {
            const size_t p = size_t(s.x) * hd->plane + size_t(s.y) * hd->pz + s.z;
            float f1 = 0, f2 = 0;
            FD_CUDA(cudaMemcpyAsync(&f1, hd->f1 + p, sizeof(float), cudaMemcpyDeviceToHost, hd->stream));
            FD_CUDA(cudaMemcpyAsync(&f2, hd->f2 + p, sizeof(float), cudaMemcpyDeviceToHost, hd->stream));
            FD_CUDA(cudaStreamSynchronize(hd->stream));
            const double w = hd->opt.form == kExpanded ? hd->dt * hd->dt / (f1 + 0.5 * hd->dt * f2) : f1;
            double qmax = 0.0;
            for (float q : s.wavelet) qmax = std::max(qmax, std::fabs(double(q)));
            bound += std::fabs(w) * qmax;
        }
    }
    hd->src_bound = float(bound);
    return FD_OK;
}

// Model upload and set-up, all O(n) work on the device: copy m (and eta) into the
// handle's fields, validate and reduce min(m) in one pass, check stability,
// build the default damping when eta is absent, then derive the factored
// form's per-point coefficients. On failure the handle has no model until a
// valid one is set.
int set_model_common(fd_handle *hd, const float *m, const float *eta, cudaMemcpyKind kind) {
    if (hd->slab && !eta)
        return fail(FD_EINVAL, "a slab needs an explicit eta (the default profile depends on the whole model)");
    hd->has_model = false;
    const size_t row_bytes = size_t(hd->Nz) * sizeof(float);
    const size_t pitch = size_t(hd->pz) * sizeof(float);
    const size_t rows = size_t(hd->Nx) * hd->Ny;
    FD_CUDA(cudaMemcpy2DAsync(hd->f1, pitch, m, row_bytes, row_bytes, rows, kind, hd->stream));
    if (eta) FD_CUDA(cudaMemcpy2DAsync(hd->f2, pitch, eta, row_bytes, row_bytes, rows, kind, hd->stream));
    const ModelCheck init{0u, 0u, 0x7f800000u, 0u};
    FD_CUDA(cudaMemcpyAsync(hd->d_check, &init, sizeof init, cudaMemcpyHostToDevice, hd->stream));
    FD_CUDA(launch_model_check(hd->f1, eta ? hd->f2 : nullptr, hd->Nx, hd->Ny, hd->Nz, hd->pz, hd->nbl,
                               hd->x_off, hd->Nx_glob, hd->d_check, hd->stream));
    ModelCheck chk;
    FD_CUDA(cudaMemcpyAsync(&chk, hd->d_check, sizeof chk, cudaMemcpyDeviceToHost, hd->stream));
    FD_CUDA(cudaStreamSynchronize(hd->stream));
    if (chk.bad_m) return fail(FD_EINVAL, "m must be positive and finite everywhere");
    if (chk.bad_eta) return fail(FD_EINVAL, "eta must be non-negative and finite everywhere");
    float mmin;
    std::memcpy(&mmin, &chk.min_m_bits, sizeof mmin);
    const double vmax = 1.0 / std::sqrt(double(mmin));
    const double dtm = stability_limit(hd->k, hd->h, vmax);
    if (hd->dt > dtm)
        return fail(FD_EUNSTABLE, "dt = %g exceeds the stability limit %g for v_max = %g", hd->dt, dtm, vmax);
    bool interior_zero = true;
    if (!eta) {
        const double dmax = hd->nbl > 0 ? 3.0 * vmax * std::log(1000.0) / (2.0 * double(hd->nbl) * hd->h) : 0.0;
        FD_CUDA(launch_default_damping(hd->f1, hd->f2, hd->Nx, hd->Ny, hd->Nz, hd->pz, hd->nbl, float(dmax),
                                       hd->stream));
    } else {
        interior_zero = chk.eta_interior_nonzero == 0;
    }
    const int lo = hd->nbl;
    if (interior_zero) {
        // the interior box in local planes (a slab sees a window of the domain's planes)
        const int bx0 = std::max(0, lo - hd->x_off), bx1 = std::min(hd->Nx, hd->Nx_glob - lo - hd->x_off);
        const int b[6] = {bx0, std::max(bx0, bx1), lo, hd->Ny - lo, lo, hd->Nz - lo};
        std::memcpy(hd->box, b, sizeof b);
    } else {
        std::memset(hd->box, 0, sizeof hd->box);
    }
    if (hd->opt.form == kFactored)
        FD_CUDA(launch_prepare_factored(hd->f1, hd->f2, (long long)hd->n_pitched, float(0.5 * hd->dt),
                                        float(hd->dt * hd->dt), hd->stream));
    FD_CUDA(cudaStreamSynchronize(hd->stream));
    hd->has_model = true;
    hd->gen++;
    return update_src_bound(hd);
}

// Level 0 (u^n) or 1 (u^{n-1}) as dense FP32 into a device buffer.
cudaError_t unpack_to(fd_handle *hd, int level, float *dst) {
    const int slot = int(((hd->step % 3) + 3) % 3);
    if (hd->opt.storage == kF32)
        return launch_unpack_level(hd->ubuf[level == 0 ? hd->cur : hd->cur ^ 1], dst, hd->Nx, hd->Ny, hd->Nz,
                                   hd->pz, kF32, nullptr, slot, hd->stream);
    if (level == 0)
        return launch_unpack_level(hd->ubuf[hd->cur], dst, hd->Nx, hd->Ny, hd->Nz, hd->pz, hd->opt.storage,
                                   hd->d_scales, slot, hd->stream);
    return launch_unpack_prev(hd->ubuf[hd->cur], hd->dbuf, dst, hd->Nx, hd->Ny, hd->Nz, hd->pz, hd->opt.storage,
                              hd->d_scales, slot, hd->stream);
}

// Trilinear cell of a continuous domain coordinate t on an axis of n >= 2
// nodes: lower node i0 = min(floor(t), n - 2) and fraction t - i0 (t in [0, n-1]).
void trilinear_axis(double t, int n, int *i0, double *f) {
    int i = int(std::floor(t));
    if (i > n - 2) i = n - 2;
    if (i < 0) i = 0;
    *i0 = i;
    *f = t - double(i);
}

bool interior_point_ok(const fd_handle *hd, double x, double y, double z) {
    return std::isfinite(x) && std::isfinite(y) && std::isfinite(z) && x >= 0.0 && y >= 0.0 && z >= 0.0 &&
           x <= double(hd->nx - 1) && y <= double(hd->ny - 1) && z <= double(hd->nz - 1);
}

// The 8 nodes (domain indices) and weights of an interior point (x, y, z).
void trilinear_nodes(const fd_handle *hd, double x, double y, double z, int nodes[8][3], double w[8]) {
    const double p[3] = {x + hd->nbl, y + hd->nbl, z + hd->nbl};
    const int n[3] = {hd->Nx, hd->Ny, hd->Nz};
    int i0[3];
    double f[3];
    for (int a = 0; a < 3; ++a) trilinear_axis(p[a], n[a], &i0[a], &f[a]);
    int c = 0;
    for (int dx = 0; dx < 2; ++dx)
        for (int dy = 0; dy < 2; ++dy)
            for (int dz = 0; dz < 2; ++dz, ++c) {
                nodes[c][0] = i0[0] + dx;
                nodes[c][1] = i0[1] + dy;
                nodes[c][2] = i0[2] + dz;
                w[c] = (dx ? f[0] : 1.0 - f[0]) * (dy ? f[1] : 1.0 - f[1]) * (dz ? f[2] : 1.0 - f[2]);
            }
}

// Free a handle's device memory in the order of its stream (after the work
// already queued there) and its host resources, without waiting for the device.
void release_handle(fd_handle *hd) {
    for (auto &g : hd->graphs)
        if (g.exec) cudaGraphExecDestroy(g.exec);
    hd->graphs.clear();
    cudaStream_t st = hd->stream ? hd->stream : hd->own_stream;
    void *bufs[] = {hd->ubuf[0], hd->ubuf[1], hd->dbuf, hd->f1, hd->f2, hd->d_wavelet, hd->d_src,
                    hd->d_status, hd->d_scales, hd->d_check, hd->d_unpack, hd->d_rec_off, hd->d_rec_w,
                    hd->d_traces, hd->tb_buf[0], hd->tb_buf[1], hd->flow_buf, hd->d_flow_tab};
    for (void *p : bufs) dev_free(p, st);
    if (hd->ev0) cudaEventDestroy(hd->ev0);
    if (hd->ev1) cudaEventDestroy(hd->ev1);
    if (hd->own_stream) cudaStreamDestroy(hd->own_stream);  // released once its work completes
    delete hd;
}

int read_status(fd_handle *hd) {
    unsigned st = 0;
    FD_CUDA(cudaMemcpyAsync(&st, hd->d_status, sizeof st, cudaMemcpyDeviceToHost, hd->stream));
    FD_CUDA(cudaStreamSynchronize(hd->stream));
    if (st & kStatusTimeout) return fail(FD_ETIMEOUT, "a device-side wait timed out (bulk copy never landed)");
    if (st & kStatusNonFinite) return fail(FD_ENONFINITE, "wavefield reached NaN/Inf (or 16-bit overflow)");
    return FD_OK;
}

}  // namespace

extern "C" {

int fd_forward_two_step(fd_handle *hd, int nt);

void fd_options_default(fd_options *opt) {
    if (!opt) return;
    opt->storage = FD_STORAGE_F32;
    opt->form = FD_FORM_FACTORED;
    opt->kernel = FD_KERNEL_AUTO;
    opt->tile_z = 0;
    opt->tile_y = 0;
    opt->x_block = 0;
    opt->check_finite = 1;
    opt->boundary = FD_BOUNDARY_ZERO;
    opt->rows = 0;
}

const char *fd_last_error(void) { return g_last_error.c_str(); }

const char *fd_version(void) { return "fdgb 0.1 (sm_103a)"; }

int fd_fd_weights(int space_order, double *out) {
    if (!out) return fail(FD_EINVAL, "out is NULL");
    if (!fornberg_second_derivative(space_order, out))
        return fail(FD_EINVAL, "space_order must be even in [2, %d], got %d", 2 * kMaxRadiusHost, space_order);
    return FD_OK;
}

int fd_default_damping(int Nx, int Ny, int Nz, int nbl, double h, const float *m, float *eta) {
    if (!m || !eta) return fail(FD_EINVAL, "m or eta is NULL");
    if (Nx < 1 || Ny < 1 || Nz < 1 || nbl < 0 || !(h > 0)) return fail(FD_EINVAL, "bad extents, nbl or h");
    const size_t n = size_t(Nx) * Ny * Nz;
    double mmin = INFINITY;
    for (size_t i = 0; i < n; ++i) {
        if (!(m[i] > 0.0f) || !std::isfinite(m[i])) return fail(FD_EINVAL, "m[%zu] is not positive finite", i);
        mmin = std::min(mmin, double(m[i]));
    }
    default_damping(m, eta, Nx, Ny, Nz, nbl, h, 1.0 / std::sqrt(mmin));
    return FD_OK;
}

int fd_dt_max(int space_order, double h, double vmax, double *out) {
    if (!out) return fail(FD_EINVAL, "out is NULL");
    const double v = stability_limit(space_order, h, vmax);
    if (!(v > 0)) return fail(FD_EINVAL, "bad space_order/h/vmax");
    *out = v;
    return FD_OK;
}

static int create_handle(int nx, int ny, int nz, int space_order, double h, double dt, int nbl,
                         const fd_options *opt_in, int slab_x0, int slab_x1, fd_handle **out);

int fd_acoustic_create_ex(int nx, int ny, int nz, int space_order, double h, double dt, int nbl,
                          const fd_options *opt_in, fd_handle **out) {
    return create_handle(nx, ny, nz, space_order, h, dt, nbl, opt_in, -1, -1, out);
}

// A whole shot (slab_x0 < 0) or the slab of planes [slab_x0, slab_x1) of it.
static int create_handle(int nx, int ny, int nz, int space_order, double h, double dt, int nbl,
                         const fd_options *opt_in, int slab_x0, int slab_x1, fd_handle **out) {
    if (!out) return fail(FD_EINVAL, "out is NULL");
    *out = nullptr;
    fd_options opt;
    fd_options_default(&opt);
    if (opt_in) opt = *opt_in;
    if (space_order < 2 || space_order > 2 * kMaxRadius || space_order % 2)
        return fail(FD_EINVAL, "space_order must be even in [2, 24], got %d", space_order);
    if (nx < 1 || ny < 1 || nz < 1 || nbl < 0)
        return fail(FD_EINVAL, "interior sizes must be >= 1 and nbl >= 0");
    if (!(h > 0) || !std::isfinite(h) || !(dt > 0) || !std::isfinite(dt))
        return fail(FD_EINVAL, "h and dt must be positive and finite");
    const long long Nx = nx + 2LL * nbl, Ny = ny + 2LL * nbl, Nz = nz + 2LL * nbl;
    if (Nx > kMaxDim || Ny > kMaxDim || Nz > kMaxDim) return fail(FD_EINVAL, "extent above 65535");
    if (opt.storage < 0 || opt.storage > 2 || opt.form < 0 || opt.form > 1 || opt.kernel < 0 ||
        opt.kernel > 3 || (opt.boundary != FD_BOUNDARY_ZERO && opt.boundary != FD_BOUNDARY_PERIODIC))
        return fail(FD_ENOTSUP, "unknown storage/form/kernel/boundary option");
    int kernel = opt.kernel;
    if (opt.boundary == FD_BOUNDARY_PERIODIC) {
        // test mode: the naive kernel with wrapped tap indices, FP32
        if (opt.storage != kF32) return fail(FD_ENOTSUP, "the periodic boundary runs on FP32 storage");
        if (kernel != kAuto && kernel != kNaive) return fail(FD_ENOTSUP, "the periodic boundary runs on the naive kernel");
        kernel = kNaive;
    }
    if (opt.storage != kF32) {
        // 16-bit storage is the increment form, computed by the TMA kernel, factored form
        if (opt.form != kFactored) return fail(FD_ENOTSUP, "16-bit storage needs the factored form");
        if (kernel != kAuto && kernel != kTma) return fail(FD_ENOTSUP, "16-bit storage runs on the TMA kernel");
    }
    if (kernel == kAuto) kernel = kTma;
    if (opt.rows < 0 || opt.rows > 2) return fail(FD_EINVAL, "rows must be 0, 1 or 2");
    if (!tile_ok(kernel, opt.storage, opt.form, space_order / 2, opt.tile_z, opt.tile_y, opt.rows))
        return fail(FD_ENOTSUP, "tile %dx%d with %d rows per thread is not a shape of the chosen kernel", opt.tile_z,
                    opt.tile_y, opt.rows);
    if (opt.x_block < 0) return fail(FD_EINVAL, "x_block must be >= 0");
    const bool slab = slab_x0 >= 0;
    int ghost_lo = 0, ghost_hi = 0;
    if (slab) {
        if (opt.storage != kF32) return fail(FD_ENOTSUP, "slabs use FP32 storage (16-bit scales are per shot)");
        if (kernel != kTma || opt.boundary != FD_BOUNDARY_ZERO)
            return fail(FD_ENOTSUP, "slabs run on the TMA kernel with the zero boundary");
        if (slab_x1 > Nx || slab_x1 - slab_x0 < space_order / 2)
            return fail(FD_EINVAL, "slab planes [%d, %d) must lie in [0, %lld) and number at least k/2 = %d",
                        slab_x0, slab_x1, Nx, space_order / 2);
        ghost_lo = slab_x0 > 0 ? space_order / 2 : 0;
        ghost_hi = slab_x1 < Nx ? space_order / 2 : 0;
    }

    fd_handle *hd = new fd_handle();
    hd->nx = nx;
    hd->ny = ny;
    hd->nz = nz;
    hd->nbl = nbl;
    hd->k = space_order;
    hd->r = space_order / 2;
    hd->h = h;
    hd->dt = dt;
    hd->Nx = int(Nx);
    hd->Ny = int(Ny);
    hd->Nz = int(Nz);
    hd->Nx_glob = int(Nx);
    hd->x_hi = int(Nx);
    if (slab) {
        hd->slab = true;
        hd->ghost_lo = ghost_lo;
        hd->ghost_hi = ghost_hi;
        hd->x_off = slab_x0 - ghost_lo;
        hd->Nx = (slab_x1 - slab_x0) + ghost_lo + ghost_hi;
        hd->x_lo = ghost_lo;
        hd->x_hi = ghost_lo + (slab_x1 - slab_x0);
    }
    hd->opt = opt;
    hd->kernel = kernel;
    hd->pz = int((Nz + 63) / 64 * 64);  // 128-byte rows for 16-bit and 256-byte rows for FP32
    hd->plane = (long long)hd->Ny * hd->pz;
    hd->n_pitched = size_t(hd->Nx) * size_t(hd->plane);
    fornberg_second_derivative(space_order, hd->coef_c);

    auto bail = [&](int code, const char *msg) {
        fd_destroy(hd);
        return fail(code, "%s", msg);
    };
    if (cudaGetDevice(&hd->device) != cudaSuccess) return bail(FD_ECUDA, "no current CUDA device");
    if (cudaStreamCreateWithFlags(&hd->own_stream, cudaStreamNonBlocking) != cudaSuccess)
        return bail(FD_ECUDA, "cudaStreamCreate failed");
    hd->stream = hd->own_stream;
    if (cudaEventCreate(&hd->ev0) != cudaSuccess || cudaEventCreate(&hd->ev1) != cudaSuccess)
        return bail(FD_ECUDA, "cudaEventCreate failed");
    const size_t ub = hd->n_pitched * elem_size(opt.storage), fb = hd->n_pitched * sizeof(float);
    cudaStream_t st = hd->stream;
    if (dev_alloc(&hd->ubuf[0], ub, st) != cudaSuccess || dev_alloc(&hd->ubuf[1], ub, st) != cudaSuccess ||
        (opt.storage != kF32 && dev_alloc(&hd->dbuf, ub, st) != cudaSuccess) ||
        dev_alloc(reinterpret_cast<void **>(&hd->f1), fb, st) != cudaSuccess ||
        dev_alloc(reinterpret_cast<void **>(&hd->f2), fb, st) != cudaSuccess ||
        dev_alloc(reinterpret_cast<void **>(&hd->d_status), sizeof(unsigned), st) != cudaSuccess ||
        dev_alloc(reinterpret_cast<void **>(&hd->d_scales), sizeof(LevelScales), st) != cudaSuccess ||
        dev_alloc(reinterpret_cast<void **>(&hd->d_check), sizeof(ModelCheck), st) != cudaSuccess) {
        cudaGetLastError();
        return bail(FD_ENOMEM, "device allocation failed");
    }
    if (cudaMemsetAsync(hd->f1, 0, fb, hd->stream) != cudaSuccess ||
        cudaMemsetAsync(hd->f2, 0, fb, hd->stream) != cudaSuccess)
        return bail(FD_ECUDA, "cudaMemset failed");
    int rc = fd_reset(hd);
    if (rc != FD_OK) {
        std::string msg = g_last_error;
        fd_destroy(hd);
        return fail(rc, "%s", msg.c_str());
    }
    *out = hd;
    return FD_OK;
}

int fd_acoustic_create(int nx, int ny, int nz, int space_order, double h, double dt, int nbl,
                       fd_handle **out) {
    return fd_acoustic_create_ex(nx, ny, nz, space_order, h, dt, nbl, nullptr, out);
}

int fd_set_model(fd_handle *hd, const float *m, const float *eta) {
    if (!hd || !m) return fail(FD_EINVAL, "handle or m is NULL");
    return set_model_common(hd, m, eta, cudaMemcpyHostToDevice);
}

int fd_set_model_device(fd_handle *hd, const float *d_m, const float *d_eta) {
    if (!hd || !d_m) return fail(FD_EINVAL, "handle or m is NULL");
    return set_model_common(hd, d_m, d_eta, cudaMemcpyDeviceToDevice);
}

int fd_inject(fd_handle *hd, int ix, int iy, int iz, const float *wavelet, int nt) {
    if (!hd) return fail(FD_EINVAL, "handle is NULL");
    if (!wavelet || nt < 1) return fail(FD_EINVAL, "wavelet is NULL or nt < 1");
    if (ix < 0 || ix >= hd->nx || iy < 0 || iy >= hd->ny || iz < 0 || iz >= hd->nz)
        return fail(FD_ERANGE, "source (%d,%d,%d) outside the %dx%dx%d interior", ix, iy, iz, hd->nx,
                    hd->ny, hd->nz);
    for (int i = 0; i < nt; ++i)
        if (!std::isfinite(wavelet[i])) return fail(FD_EINVAL, "wavelet[%d] is not finite", i);
    const int lx = ix + hd->nbl - hd->x_off;  // local plane (a slab keeps only its own planes' sources)
    if (hd->slab && (lx < hd->x_lo || lx >= hd->x_hi)) return FD_OK;
    if (hd->slab && int(hd->sources.size()) >= kFusedSources)
        return fail(FD_ENOTSUP, "a slab takes at most %d sources in its planes", kFusedSources);
    Source s{lx, iy + hd->nbl, iz + hd->nbl, std::vector<float>(wavelet, wavelet + nt)};
    hd->sources.push_back(std::move(s));
    int rc = upload_sources(hd);
    if (rc != FD_OK) {
        hd->sources.pop_back();
        return rc;
    }
    hd->gen++;
    return update_src_bound(hd);
}

int fd_inject_at(fd_handle *hd, double x, double y, double z, const float *wavelet, int nt) {
    if (!hd) return fail(FD_EINVAL, "handle is NULL");
    if (hd->slab) return fail(FD_ENOTSUP, "slabs take integer-node sources and no receivers");
    if (!wavelet || nt < 1) return fail(FD_EINVAL, "wavelet is NULL or nt < 1");
    if (!interior_point_ok(hd, x, y, z))
        return fail(FD_ERANGE, "source (%g,%g,%g) outside the [0,%d]x[0,%d]x[0,%d] interior", x, y, z, hd->nx - 1,
                    hd->ny - 1, hd->nz - 1);
    for (int i = 0; i < nt; ++i)
        if (!std::isfinite(wavelet[i])) return fail(FD_EINVAL, "wavelet[%d] is not finite", i);
    int nodes[8][3];
    double w[8];
    trilinear_nodes(hd, x, y, z, nodes, w);
    const size_t before = hd->sources.size();
    for (int c = 0; c < 8; ++c) {
        if (w[c] <= 0.0) continue;
        Source s{nodes[c][0], nodes[c][1], nodes[c][2], std::vector<float>(size_t(nt))};
        for (int i = 0; i < nt; ++i) s.wavelet[size_t(i)] = float(w[c] * double(wavelet[i]));
        hd->sources.push_back(std::move(s));
    }
    int rc = upload_sources(hd);
    if (rc != FD_OK) {
        hd->sources.resize(before);
        return rc;
    }
    hd->gen++;
    return update_src_bound(hd);
}

int fd_set_receivers(fd_handle *hd, int n, const double *xyz, int nt_max) {
    if (!hd) return fail(FD_EINVAL, "handle is NULL");
    if (hd->slab) return fail(FD_ENOTSUP, "slabs take integer-node sources and no receivers");
    if (n < 0 || (n > 0 && (!xyz || nt_max < 1))) return fail(FD_EINVAL, "bad receiver count, positions or nt_max");
    if (n > 0 && (long long)n * nt_max > (1LL << 31))
        return fail(FD_EINVAL, "n * nt_max above 2^31 samples");
    for (int r = 0; r < n; ++r)
        if (!interior_point_ok(hd, xyz[3 * r], xyz[3 * r + 1], xyz[3 * r + 2]))
            return fail(FD_ERANGE, "receiver %d (%g,%g,%g) outside the interior", r, xyz[3 * r], xyz[3 * r + 1],
                        xyz[3 * r + 2]);
    // queued steps may still write the old traces: the old arrays are freed behind them
    dev_free(hd->d_rec_off, hd->stream);
    dev_free(hd->d_rec_w, hd->stream);
    dev_free(hd->d_traces, hd->stream);
    hd->d_rec_off = nullptr;
    hd->d_rec_w = nullptr;
    hd->d_traces = nullptr;
    hd->n_rec = 0;
    hd->rec_nt_max = 0;
    hd->rec_node.clear();
    hd->rec_off_h.clear();
    hd->rec_w_h.clear();
    hd->gen++;
    if (n == 0) return FD_OK;
    std::vector<long long> off(size_t(n) * 8);
    std::vector<float> w(size_t(n) * 8);
    std::vector<int> lower(size_t(n) * 3);
    for (int r = 0; r < n; ++r) {
        int nodes[8][3];
        double wd[8];
        trilinear_nodes(hd, xyz[3 * r], xyz[3 * r + 1], xyz[3 * r + 2], nodes, wd);
        for (int a = 0; a < 3; ++a) lower[size_t(r) * 3 + a] = nodes[0][a];
        for (int c = 0; c < 8; ++c) {
            off[size_t(r) * 8 + c] = (long long)nodes[c][0] * hd->plane + (long long)nodes[c][1] * hd->pz + nodes[c][2];
            w[size_t(r) * 8 + c] = float(wd[c]);
        }
    }
    const size_t nsamp = size_t(n) * size_t(nt_max);
    if (dev_alloc(reinterpret_cast<void **>(&hd->d_rec_off), off.size() * sizeof(long long), hd->stream) != cudaSuccess ||
        dev_alloc(reinterpret_cast<void **>(&hd->d_rec_w), w.size() * sizeof(float), hd->stream) != cudaSuccess ||
        dev_alloc(reinterpret_cast<void **>(&hd->d_traces), nsamp * sizeof(float), hd->stream) != cudaSuccess) {
        cudaGetLastError();
        dev_free(hd->d_rec_off, hd->stream);
        dev_free(hd->d_rec_w, hd->stream);
        dev_free(hd->d_traces, hd->stream);
        hd->d_rec_off = nullptr;
        hd->d_rec_w = nullptr;
        hd->d_traces = nullptr;
        return fail(FD_ENOMEM, "cannot allocate receivers");
    }
    FD_CUDA(cudaMemcpyAsync(hd->d_rec_off, off.data(), off.size() * sizeof(long long), cudaMemcpyHostToDevice,
                            hd->stream));
    FD_CUDA(cudaMemcpyAsync(hd->d_rec_w, w.data(), w.size() * sizeof(float), cudaMemcpyHostToDevice, hd->stream));
    FD_CUDA(cudaMemsetAsync(hd->d_traces, 0, nsamp * sizeof(float), hd->stream));
    FD_CUDA(cudaStreamSynchronize(hd->stream));  // the host vectors go out of scope
    hd->n_rec = n;
    hd->rec_nt_max = nt_max;
    hd->rec_step0 = hd->step;
    hd->rec_node = std::move(lower);
    hd->rec_off_h = std::move(off);
    hd->rec_w_h = std::move(w);
    return FD_OK;
}

int fd_read_traces(fd_handle *hd, float *out, int *recorded) {
    if (!hd || !out || !recorded) return fail(FD_EINVAL, "NULL argument");
    if (hd->n_rec == 0) return fail(FD_ESTATE, "no receivers set");
    const long long done = std::max(0LL, std::min<long long>(hd->step - hd->rec_step0, hd->rec_nt_max));
    FD_CUDA(cudaMemcpyAsync(out, hd->d_traces, size_t(hd->n_rec) * hd->rec_nt_max * sizeof(float),
                            cudaMemcpyDeviceToHost, hd->stream));
    FD_CUDA(cudaStreamSynchronize(hd->stream));
    *recorded = int(done);
    return check_enabled(hd) ? read_status(hd) : FD_OK;
}

// The FWI gradient (see fd_fwi_gradient in the header). segment >= nt keeps the
// second time difference of every step in device memory; a shorter segment
// keeps only the states (u^j, u^{j-1}) at every segment-th step during the
// forward pass and, during the adjoint pass, recomputes each segment's
// history from its checkpoint (one extra forward pass; memory ~ 2 nt/segment +
// segment fields). The recomputation uses the same per-point arithmetic, so
// both give the same bits.
static int fwi_gradient_impl(fd_handle *hd, int nrec, const double *rec_xyz, const float *d_obs, int nt,
                             int segment, float *grad_out, float *syn_out, double *misfit) {
    if (!hd || nrec < 1 || !rec_xyz || !d_obs || nt < 1 || !grad_out || !misfit || segment < 0)
        return fail(FD_EINVAL, "bad receivers, data, nt, segment or output pointers");
    if (hd->slab) return fail(FD_ENOTSUP, "the FWI gradient runs on whole shots, not slabs");
    if (!hd->has_model) return fail(FD_ESTATE, "fd_fwi_gradient before fd_set_model");
    if (hd->opt.storage != kF32 || hd->opt.form != kFactored || hd->kernel != kTma)
        return fail(FD_ENOTSUP, "the FWI gradient runs on FP32 storage, factored form, TMA kernel");
    if ((long long)nrec * nt > (1LL << 31)) return fail(FD_EINVAL, "nrec * nt above 2^31 samples");
    for (int r = 0; r < nrec; ++r)
        if (!interior_point_ok(hd, rec_xyz[3 * r], rec_xyz[3 * r + 1], rec_xyz[3 * r + 2]))
            return fail(FD_ERANGE, "receiver %d outside the interior", r);
    if (hd->tile_y == 0 || hd->x_block == 0) {  // the plain steps of the checkpointed pass use the tuned shape
        int rc = autotune(hd);
        if (rc == FD_OK) rc = build_maps(hd);
        if (rc != FD_OK) {
            hd->tile_y = hd->x_block = 0;
            return rc;
        }
        hd->gen++;
    }
    cudaStream_t st = hd->stream;
    const size_t np = hd->n_pitched;
    const size_t fbytes = np * sizeof(float);
    if (segment == 0) {
        // automatic: the full history if it fits in 80 % of the free memory, else segments of sqrt(nt)
        size_t free_b = 0, total_b = 0;
        cudaMemGetInfo(&free_b, &total_b);
        const double need = double(nt + 4) * double(fbytes) + double(nrec) * nt * 8.0;
        segment = need <= 0.8 * double(free_b) ? nt : std::max(1, int(std::ceil(std::sqrt(double(nt)))));
    }
    segment = std::min(segment, nt);
    const int nseg = (nt + segment - 1) / segment;
    const bool ckpt = nseg > 1;
    const int tz = 32, ty = 16;  // the gradient passes' tile
    const int xb = (hd->tile_z == tz && hd->tile_y == ty && hd->x_block > 0) ? hd->x_block
                                                                              : heuristic_x_block(hd, tz, ty);
    // workspace: the history of one segment (all steps without checkpoints), the
    // checkpoints, the gradient, two adjoint fields, the residuals, the receivers' node lists
    float *hist = nullptr, *ckp = nullptr, *grad = nullptr, *w[2] = {nullptr, nullptr}, *resid = nullptr;
    long long *node_off = nullptr;
    int *row = nullptr, *rec_idx = nullptr;
    float *rec_w = nullptr;
    auto release = [&]() {
        void *bufs[] = {hist, ckp, grad, w[0], w[1], resid, node_off, row, rec_idx, rec_w};
        for (void *p : bufs) dev_free(p, st);
    };
    // the receivers' spreading as a node-major list (fixed order within a node)
    struct Entry {
        long long off;
        int rec;
        float w;
    };
    std::vector<Entry> ent;
    for (int r = 0; r < nrec; ++r) {
        int nodes[8][3];
        double wd[8];
        trilinear_nodes(hd, rec_xyz[3 * r], rec_xyz[3 * r + 1], rec_xyz[3 * r + 2], nodes, wd);
        for (int c = 0; c < 8; ++c)
            if (wd[c] > 0.0)
                ent.push_back({(long long)nodes[c][0] * hd->plane + (long long)nodes[c][1] * hd->pz + nodes[c][2], r,
                               float(wd[c])});
    }
    std::stable_sort(ent.begin(), ent.end(), [](const Entry &a, const Entry &b) { return a.off < b.off; });
    std::vector<long long> h_node;
    std::vector<int> h_row, h_rec;
    std::vector<float> h_w;
    for (size_t e = 0; e < ent.size(); ++e) {
        if (e == 0 || ent[e].off != ent[e - 1].off) {
            h_node.push_back(ent[e].off);
            h_row.push_back(int(e));
        }
        h_rec.push_back(ent[e].rec);
        h_w.push_back(ent[e].w);
    }
    h_row.push_back(int(ent.size()));
    const int n_nodes = int(h_node.size());
    if (dev_alloc(reinterpret_cast<void **>(&hist), size_t(segment) * fbytes, st) != cudaSuccess ||
        (ckpt && dev_alloc(reinterpret_cast<void **>(&ckp), size_t(2 * nseg) * fbytes, st) != cudaSuccess) ||
        dev_alloc(reinterpret_cast<void **>(&grad), fbytes, st) != cudaSuccess ||
        dev_alloc(reinterpret_cast<void **>(&w[0]), fbytes, st) != cudaSuccess ||
        dev_alloc(reinterpret_cast<void **>(&w[1]), fbytes, st) != cudaSuccess ||
        dev_alloc(reinterpret_cast<void **>(&resid), size_t(nrec) * nt * sizeof(float), st) != cudaSuccess ||
        dev_alloc(reinterpret_cast<void **>(&node_off), h_node.size() * sizeof(long long), st) != cudaSuccess ||
        dev_alloc(reinterpret_cast<void **>(&row), h_row.size() * sizeof(int), st) != cudaSuccess ||
        dev_alloc(reinterpret_cast<void **>(&rec_idx), h_rec.size() * sizeof(int), st) != cudaSuccess ||
        dev_alloc(reinterpret_cast<void **>(&rec_w), h_w.size() * sizeof(float), st) != cudaSuccess) {
        cudaGetLastError();
        release();
        return fail(FD_ENOMEM, "cannot allocate the gradient workspace (%d history levels, %d checkpoints)", segment,
                    ckpt ? nseg : 0);
    }
    auto cuda_fail = [&](cudaError_t e) {
        release();
        return fail(FD_ECUDA, "fd_fwi_gradient: %s", cudaGetErrorString(e));
    };
    // d_obs goes to the residual buffer now; the residual is formed on the device after
    // the forward pass, so that the passes run back to back
    cudaError_t e = cudaMemcpyAsync(resid, d_obs, size_t(nrec) * nt * sizeof(float), cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(node_off, h_node.data(), h_node.size() * sizeof(long long), cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(row, h_row.data(), h_row.size() * sizeof(int), cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(rec_idx, h_rec.data(), h_rec.size() * sizeof(int), cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(rec_w, h_w.data(), h_w.size() * sizeof(float), cudaMemcpyHostToDevice, st);
    if (e != cudaSuccess) return cuda_fail(e);
    int rc = fd_reset(hd);
    if (rc == FD_OK) rc = fd_set_receivers(hd, nrec, rec_xyz, nt);
    TmaMaps fm[2], am[2];
    GradMaps gm{};
    for (int b = 0; b < 2 && rc == FD_OK; ++b) rc = make_maps(hd, hd->ubuf[b], hd->ubuf[b ^ 1], tz, ty, 1, &fm[b]);
    for (int b = 0; b < 2 && rc == FD_OK; ++b) rc = make_maps(hd, w[b], w[b ^ 1], tz, ty, 1, &am[b]);
    if (rc == FD_OK) rc = encode_box(hd, grad, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 4, tz, ty, &gm.grad);
    if (rc == FD_OK) {
        // the history as one 4-D tensor: level k - 1 of step k is the fourth coordinate
        EncodeTiledFn fn = encode_fn();
        cuuint64_t dims[4] = {cuuint64_t(hd->Nz), cuuint64_t(hd->Ny), cuuint64_t(hd->Nx), cuuint64_t(segment)};
        cuuint64_t strides[3] = {cuuint64_t(hd->pz) * 4, cuuint64_t(hd->plane) * 4, cuuint64_t(np) * 4};
        cuuint32_t box[4] = {cuuint32_t(tz), cuuint32_t(ty), 1, 1};
        cuuint32_t estr[4] = {1, 1, 1, 1};
        if (!fn || fn(&gm.hist, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 4, hist, dims, strides, box, estr,
                      CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
                      CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
            rc = fail(FD_ECUDA, "cuTensorMapEncodeTiled failed for the history");
    }
    if (rc != FD_OK) {
        release();
        return rc;
    }
    const bool check = check_enabled(hd);
    const int ns = int(hd->sources.size());
    // forward steps [n0, n1) from the handle's fields (cur), storing D^n at hist[n - n0]
    // (with_receivers: the traces of those steps are recorded)
    auto forward_d = [&](int n0, int n1, int &cur, bool with_receivers) {
        cudaError_t err = cudaSuccess;
        for (int n = n0; n < n1 && err == cudaSuccess; ++n) {
            StepArgs a = make_args(hd, n, cur);
            a.x_block = xb;
            a.hist = hist + size_t(n - n0) * np;
            if (!with_receivers) {
                a.n_rec = 0;
                a.rec_sample = -1;
            }
            err = launch_tma_grad_step(hd->r, kModeForwardD, fm[cur], gm, a, check, st);
            if (err == cudaSuccess && ns > kFusedSources)
                err = launch_inject_extra(a, hd->d_src, hd->d_src + ns, hd->d_src + 2 * ns, kFusedSources,
                                          ns - kFusedSources, kF32, 0, hd->extra_distinct, st, a.hist);
            cur ^= 1;
        }
        return err;
    };
    int cur = hd->cur;
    e = cudaEventRecord(hd->ev0, st);  // device time of the passes: fd_last_forward_ms
    if (!ckpt) {
        if (e == cudaSuccess) e = forward_d(0, nt, cur, true);
    } else {
        // plain steps; the states (u^j, u^{j-1}) at j = 0, segment, 2 segment, ... are kept
        for (int n = 0; n < nt && e == cudaSuccess; ++n) {
            if (n % segment == 0) {
                const size_t slot = size_t(2 * (n / segment));
                e = cudaMemcpyAsync(ckp + slot * np, hd->ubuf[cur], fbytes, cudaMemcpyDeviceToDevice, st);
                if (e == cudaSuccess)
                    e = cudaMemcpyAsync(ckp + (slot + 1) * np, hd->ubuf[cur ^ 1], fbytes, cudaMemcpyDeviceToDevice, st);
            }
            if (e == cudaSuccess) e = enqueue_step(hd, make_args(hd, n, cur), st);
            cur ^= 1;
        }
    }
    if (e == cudaSuccess) e = sample_level(hd, hd->ubuf[cur], nt, st);
    const int cur_end = cur;
    // residual r = d - d_obs (in place over d_obs)
    if (e == cudaSuccess) e = launch_residual(hd->d_traces, resid, size_t(nrec) * nt, st);
    // adjoint pass, backward in time: w^k over w^{k+2} from w^{k+1}, the residual of
    // step k-1 injected at the receivers' nodes, gradient -= w^k D^{k-1}
    if (e == cudaSuccess) e = cudaMemsetAsync(grad, 0, fbytes, st);
    if (e == cudaSuccess) e = cudaMemsetAsync(w[0], 0, fbytes, st);
    if (e == cudaSuccess) e = cudaMemsetAsync(w[1], 0, fbytes, st);
    const float inv_dt2 = float(1.0 / (hd->dt * hd->dt));
    int c = 0;  // w[c] holds w^{k+1}, w[c^1] w^{k+2}
    for (int sg = nseg - 1; sg >= 0 && e == cudaSuccess; --sg) {
        const int n0 = sg * segment, n1 = std::min(nt, n0 + segment);
        if (ckpt) {
            // recompute this segment's history from its checkpoint
            const size_t slot = size_t(2 * sg);
            int rcur = 0;
            e = cudaMemcpyAsync(hd->ubuf[0], ckp + slot * np, fbytes, cudaMemcpyDeviceToDevice, st);
            if (e == cudaSuccess)
                e = cudaMemcpyAsync(hd->ubuf[1], ckp + (slot + 1) * np, fbytes, cudaMemcpyDeviceToDevice, st);
            if (e == cudaSuccess) e = forward_d(n0, n1, rcur, false);
        }
        for (int k = n1; k > n0 && e == cudaSuccess; --k) {
            StepArgs a = make_args(hd, 0, 0);
            a.u = w[c];
            a.up = w[c ^ 1];
            a.ns = 0;
            a.n_rec = 0;
            a.rec_sample = -1;
            a.x_block = xb;
            a.hist = hist + size_t(k - 1 - n0) * np;
            a.hist_slot = k - 1 - n0;
            a.grad = grad;
            e = launch_tma_grad_step(hd->r, kModeAdjointGrad, am[c], gm, a, check, st);
            if (e == cudaSuccess)
                e = launch_adjoint_inject(w[c ^ 1], grad, a.hist, hd->f1, node_off, row, rec_idx, rec_w, resid, nt,
                                          k - 1, inv_dt2, n_nodes, st);
            c ^= 1;
        }
    }
    if (e == cudaSuccess) e = cudaEventRecord(hd->ev1, st);
    hd->timed = e == cudaSuccess;
    // the handle ends at step nt (with checkpoints its fields hold a recomputed early state:
    // the last state is restored from the end of the forward pass only without them)
    hd->step = nt;
    hd->cur = cur_end;
    if (ckpt && e == cudaSuccess) {
        // put u^nt, u^{nt-1} back: recompute the last segment's end state from its checkpoint
        const int sg = nseg - 1, n0 = sg * segment;
        const size_t slot = size_t(2 * sg);
        int rcur = 0;
        e = cudaMemcpyAsync(hd->ubuf[0], ckp + slot * np, fbytes, cudaMemcpyDeviceToDevice, st);
        if (e == cudaSuccess) e = cudaMemcpyAsync(hd->ubuf[1], ckp + (slot + 1) * np, fbytes, cudaMemcpyDeviceToDevice, st);
        for (int n = n0; n < nt && e == cudaSuccess; ++n) {
            StepArgs a = make_args(hd, n, rcur);
            a.n_rec = 0;
            a.rec_sample = -1;
            e = enqueue_step(hd, a, st);
            rcur ^= 1;
        }
        hd->cur = rcur;
    }
    // the traces (synthetic data) and the misfit (FP64 sum on the host)
    std::vector<float> syn(size_t(nrec) * nt);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(syn.data(), hd->d_traces, syn.size() * sizeof(float), cudaMemcpyDeviceToHost, st);
    const size_t row_bytes = size_t(hd->Nz) * sizeof(float);
    if (e == cudaSuccess)
        e = cudaMemcpy2DAsync(grad_out, row_bytes, grad, size_t(hd->pz) * sizeof(float), row_bytes,
                              size_t(hd->Nx) * hd->Ny, cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return cuda_fail(e);
    double J = 0.0;
    for (size_t i = 0; i < syn.size(); ++i) {
        const double d = double(syn[i]) - double(d_obs[i]);
        J += 0.5 * d * d;
    }
    if (syn_out) std::memcpy(syn_out, syn.data(), syn.size() * sizeof(float));
    *misfit = J;
    release();
    return check ? read_status(hd) : FD_OK;
}

int fd_fwi_gradient(fd_handle *hd, int nrec, const double *rec_xyz, const float *d_obs, int nt, float *grad_out,
                    float *syn_out, double *misfit) {
    return fwi_gradient_impl(hd, nrec, rec_xyz, d_obs, nt, 0, grad_out, syn_out, misfit);
}

int fd_fwi_gradient_checkpointed(fd_handle *hd, int nrec, const double *rec_xyz, const float *d_obs, int nt,
                                 int segment, float *grad_out, float *syn_out, double *misfit) {
    if (segment < 1) return fail(FD_EINVAL, "segment must be >= 1");
    return fwi_gradient_impl(hd, nrec, rec_xyz, d_obs, nt, segment, grad_out, syn_out, misfit);
}

// Tensor maps of the two-step kernel for input pair (u^n in u, u^{n-1} in up).
static int tb_maps_for(fd_handle *hd, const void *u, const void *up, const TmaMaps **out) {
    for (auto &m : hd->tb_maps)
        if (m.u == u && m.up == up) {
            *out = &m.maps;
            return FD_OK;
        }
    int tz, ty, bw, bh, ez, ey;
    if (!tma2_geometry(hd->r, &tz, &ty, &bw, &bh, &ez, &ey)) return fail(FD_ENOTSUP, "no two-step kernel");
    fd_handle::TbMaps m{u, up, {}};
    int rc = encode_box(hd, u, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 4, bw, bh, &m.maps.u_halo);
    if (rc == FD_OK) rc = encode_box(hd, u, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 4, ez, ey, &m.maps.u_pt);
    if (rc == FD_OK) rc = encode_box(hd, up, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 4, ez, ey, &m.maps.up_pt);
    if (rc == FD_OK) rc = encode_box(hd, hd->f1, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 4, ez, ey, &m.maps.f1_pt);
    if (rc == FD_OK) rc = encode_box(hd, hd->f2, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 4, ez, ey, &m.maps.f2_pt);
    if (rc != FD_OK) return rc;
    if (hd->tb_maps.size() >= 4) hd->tb_maps.erase(hd->tb_maps.begin());
    hd->tb_maps.push_back(m);
    *out = &hd->tb_maps.back().maps;
    return FD_OK;
}

int fd_forward_two_step(fd_handle *hd, int nt) {
    if (!hd) return fail(FD_EINVAL, "handle is NULL");
    if (hd->slab) return fail(FD_ENOTSUP, "a slab advances through fd_slab_step, with its halo exchange");
    if (nt < 0) return fail(FD_EINVAL, "nt must be >= 0");
    if (!hd->has_model) return fail(FD_ESTATE, "fd_forward_two_step before fd_set_model");
    if (hd->opt.storage != kF32 || hd->opt.form != kFactored || hd->r > 2 || hd->n_rec > 0 ||
        int(hd->sources.size()) > kFusedSources || hd->opt.boundary != FD_BOUNDARY_ZERO)
        return fail(FD_ENOTSUP,
                    "two steps per launch: FP32 factored, space order <= 4, <= %d sources, no receivers, zero boundary",
                    kFusedSources);
    if (nt == 0) return FD_OK;
    cudaStream_t st = hd->stream;
    const size_t ub = hd->n_pitched * sizeof(float);
    if (!hd->tb_buf[0]) {
        for (int b = 0; b < 2; ++b) {
            if (dev_alloc(&hd->tb_buf[b], ub, st) != cudaSuccess) {
                cudaGetLastError();
                return fail(FD_ENOMEM, "cannot allocate the two-step output buffers");
            }
            FD_CUDA(cudaMemsetAsync(hd->tb_buf[b], 0, ub, st));  // the pitch padding stays zero
        }
    }
    const bool check = check_enabled(hd);
    int tz, ty, bw, bh, ez, ey;
    tma2_geometry(hd->r, &tz, &ty, &bw, &bh, &ez, &ey);
    if (hd->tb_xb == 0) {
        std::lock_guard<std::mutex> lk(g_tune_mu);
        auto it = g_tb_cache.find(std::make_tuple(hd->Nx, hd->Ny, hd->Nz, hd->r));
        if (it != g_tb_cache.end()) hd->tb_xb = it->second;
    }
    if (hd->tb_xb == 0) {
        // x_block by timing candidates; the launches only write the output pair, so the state stays
        const TmaMaps *m = nullptr;
        int rc = tb_maps_for(hd, hd->ubuf[hd->cur], hd->ubuf[hd->cur ^ 1], &m);
        if (rc != FD_OK) return rc;
        int dev = 0, sms = 152;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        const long long tiles = (long long)((hd->Nz + tz - 1) / tz) * ((hd->Ny + ty - 1) / ty);
        std::vector<int> cand = {16, 24, 32, 48, 64, 96};
        for (int waves = 1; waves <= 3; ++waves) {
            const long long chunks = 2LL * sms * waves / std::max(1LL, tiles);
            if (chunks >= 1) cand.push_back(int((hd->Nx + chunks - 1) / chunks));
        }
        cand.push_back(hd->Nx);
        float best = 1e30f;
        int best_xb = hd->Nx;
        for (int xb : cand) {
            if (xb < 4 || xb > hd->Nx) continue;
            StepArgs a = make_args(hd, hd->step, hd->cur);
            a.x_block = xb;
            a.n_rec = 0;
            a.rec_sample = -1;
            a.status = nullptr;
            cudaError_t e = cudaSuccess;
            for (int w = 0; w < 1 && e == cudaSuccess; ++w)
                e = launch_tma2_step(hd->r, *m, a, static_cast<float *>(hd->tb_buf[0]),
                                     static_cast<float *>(hd->tb_buf[1]), false, st);
            if (e == cudaSuccess) e = cudaEventRecord(hd->ev0, st);
            for (int w = 0; w < 3 && e == cudaSuccess; ++w)
                e = launch_tma2_step(hd->r, *m, a, static_cast<float *>(hd->tb_buf[0]),
                                     static_cast<float *>(hd->tb_buf[1]), false, st);
            if (e == cudaSuccess) e = cudaEventRecord(hd->ev1, st);
            if (e == cudaSuccess) e = cudaEventSynchronize(hd->ev1);
            float ms = 0;
            if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, hd->ev0, hd->ev1);
            if (e != cudaSuccess) return fail(FD_ECUDA, "two-step tuning failed: %s", cudaGetErrorString(e));
            if (ms < best) {
                best = ms;
                best_xb = xb;
            }
        }
        hd->tb_xb = best_xb;
        std::lock_guard<std::mutex> lk(g_tune_mu);
        g_tb_cache[std::make_tuple(hd->Nx, hd->Ny, hd->Nz, hd->r)] = best_xb;
    }
    if (nt % 2) {
        // the odd step first, by the single-step kernel (the steps give the same bits
        // in either order); the start event it records opens this call's timed span
        int rc = fd_forward(hd, 1);
        if (rc != FD_OK) return rc;
    } else {
        FD_CUDA(cudaEventRecord(hd->ev0, st));
    }
    for (int p = 0; p + 1 < nt; p += 2) {
        const TmaMaps *m = nullptr;
        int rc = tb_maps_for(hd, hd->ubuf[hd->cur], hd->ubuf[hd->cur ^ 1], &m);
        if (rc != FD_OK) return rc;
        StepArgs a = make_args(hd, hd->step, hd->cur);
        a.x_block = hd->tb_xb;
        a.n_rec = 0;
        a.rec_sample = -1;
        FD_CUDA(launch_tma2_step(hd->r, *m, a, static_cast<float *>(hd->tb_buf[0]), static_cast<float *>(hd->tb_buf[1]),
                                 check, st));
        // the outputs become the state (u^{n+2}, u^{n+1}); the inputs the next output pair
        void *old_u = hd->ubuf[hd->cur], *old_up = hd->ubuf[hd->cur ^ 1];
        hd->ubuf[0] = hd->tb_buf[1];
        hd->ubuf[1] = hd->tb_buf[0];
        hd->tb_buf[0] = old_u;
        hd->tb_buf[1] = old_up;
        hd->cur = 0;
        hd->step += 2;
    }
    FD_CUDA(cudaEventRecord(hd->ev1, st));
    hd->timed = true;
    // the buffers moved: single-step maps and graphs refer to the old arrangement
    hd->gen++;
    if (hd->kernel == kTma && hd->tile_y > 0) {
        int rc = build_maps(hd);
        if (rc != FD_OK) return rc;
    }
    return FD_OK;
}

int fd_clear_sources(fd_handle *hd) {
    if (!hd) return fail(FD_EINVAL, "handle is NULL");
    hd->sources.clear();
    int rc = upload_sources(hd);
    hd->gen++;
    hd->src_bound = 0.0f;
    return rc;
}

// Replays the handle's CUDA graph of nt steps from its current state
// (recording it first, or updating it when only the step changed); `record`
// enqueues the steps on the capturing stream. Timed by the handle's events;
// advances the step counter and the buffer parity.
extern "C++" {
template <typename F>
int replay_graph(fd_handle *hd, int nt, bool flow, F &&record) {
    GraphEntry *entry = nullptr;
    for (auto &g : hd->graphs)
        if (g.nt == nt && g.cur == hd->cur && g.gen == hd->gen && g.flow == flow) entry = &g;
    if (!entry || entry->step0 != hd->step) {
        cudaGraph_t graph = nullptr;
        FD_CUDA(cudaStreamBeginCapture(hd->stream, cudaStreamCaptureModeThreadLocal));
        const long long captured0 = captured_launches();
        cudaError_t err = record(hd->stream);
        cudaError_t cap = cudaStreamEndCapture(hd->stream, &graph);
        if (err != cudaSuccess || cap != cudaSuccess) {
            if (graph) cudaGraphDestroy(graph);
            return fail(FD_ECUDA, "graph capture failed: %s",
                        cudaGetErrorString(err != cudaSuccess ? err : cap));
        }
        bool updated = false;
        if (entry) {
            cudaGraphExecUpdateResultInfo info;
            if (cudaGraphExecUpdate(entry->exec, graph, &info) == cudaSuccess) {
                updated = true;
            } else {
                cudaGetLastError();
                cudaGraphExecDestroy(entry->exec);
                entry->exec = nullptr;
            }
        }
        if (!updated) {
            cudaGraphExec_t exec = nullptr;
            cudaError_t ie = cudaGraphInstantiate(&exec, graph, 0);
            if (ie != cudaSuccess) {
                cudaGraphDestroy(graph);
                return fail(FD_ECUDA, "cudaGraphInstantiate failed: %s", cudaGetErrorString(ie));
            }
            if (!entry) {
                if (hd->graphs.size() >= 8) {
                    cudaStreamSynchronize(hd->stream);  // the oldest graph may still be queued
                    cudaGraphExecDestroy(hd->graphs.front().exec);
                    hd->graphs.erase(hd->graphs.begin());
                }
                hd->graphs.push_back(GraphEntry{});
                entry = &hd->graphs.back();
            }
            entry->exec = exec;
        }
        cudaGraphDestroy(graph);
        entry->launches = captured_launches() - captured0;
        entry->nt = nt;
        entry->flow = flow;
        entry->cur = hd->cur;
        entry->gen = hd->gen;
        entry->step0 = hd->step;
    }
    FD_CUDA(cudaEventRecord(hd->ev0, hd->stream));
    FD_CUDA(cudaGraphLaunch(entry->exec, hd->stream));
    count_replay(entry->launches);
    FD_CUDA(cudaEventRecord(hd->ev1, hd->stream));
    hd->timed = true;
    hd->step += nt;
    hd->cur ^= (nt & 1);
    return FD_OK;
}
}  // extern "C++"

static int ensure_step_tuned(fd_handle *hd);
static int run_steps(fd_handle *hd, int nt);
static int run_flow(fd_handle *hd, int nt);
static bool flow_eligible(const fd_handle *hd);
static int flow_prepare(fd_handle *hd, int *nt);

int fd_forward(fd_handle *hd, int nt) {
    if (!hd) return fail(FD_EINVAL, "handle is NULL");
    if (hd->slab) return fail(FD_ENOTSUP, "a slab advances through fd_slab_step, with its halo exchange");
    if (nt < 0) return fail(FD_EINVAL, "nt must be >= 0");
    if (!hd->has_model) return fail(FD_ESTATE, "fd_forward before fd_set_model");
    if (nt == 0) return FD_OK;
    // automatic kernel choice, space order 2: two steps per launch where the single-step
    // kernel is bound by HBM traffic (measured 1.15x at 276^3; at space order 4 the
    // overlap of the extended tiles costs more than the traffic saved). Same bits.
    if (nt >= 2 && hd->opt.kernel == kAuto && hd->kernel == kTma && hd->r == 1 && hd->opt.storage == kF32 &&
        hd->opt.form == kFactored && hd->n_rec == 0 && int(hd->sources.size()) <= kFusedSources)
        return fd_forward_two_step(hd, nt);
    // automatic kernel choice, FP32 otherwise: the flow schedule (one persistent launch,
    // no per-step tail or launch gap; measured 1.02-1.10x over per-step launches at
    // 276^3 for every space order and form) where it was timed faster than the per-step
    // launches for this grid. Same bits either way.
    if (hd->opt.kernel == kAuto && flow_eligible(hd)) {
        int rc = flow_prepare(hd, &nt);
        if (rc != FD_OK || nt == 0) return rc;
        return hd->flow_wins ? run_flow(hd, nt) : run_steps(hd, nt);
    }
    int rc = ensure_step_tuned(hd);
    if (rc != FD_OK) return rc;
    return run_steps(hd, nt);
}

// FP32 flow with receivers or sources beyond the fused ones: the per-region
// entry tables (regions numbered as the flow's flags: x-chunk, y tile, z tile,
// z fastest; a receiver belongs to the region of its lower corner node, a source
// to that of its node; entries of a region in receiver / source order). One
// device buffer: rec_start[P + 1], rec_row[n_rec], xs_start[P + 1],
// xs_idx[n_x], then (64-byte aligned) rec_off[n_rec] (lower corner node),
// xs_off[n_x] and rec_w[8 n_rec]. Rebuilt when the x_block or the handle's state changes; a
// rebuild re-records the graphs.
struct FlowTables {
    size_t rec_start, rec_row, xs_start, xs_idx, rec_off, xs_off, rec_w, bytes;
};

static FlowTables flow_table_layout(long long regions, int n_rec, int n_x) {
    auto up = [](size_t b, size_t a) { return (b + a - 1) / a * a; };
    FlowTables t{};
    size_t b = 0;
    t.rec_start = b;
    b += n_rec > 0 ? size_t(regions + 1) * sizeof(int) : 0;
    t.rec_row = b;
    b += size_t(n_rec) * sizeof(int);
    t.xs_start = b;
    b += n_x > 0 ? size_t(regions + 1) * sizeof(int) : 0;
    t.xs_idx = b;
    b += size_t(n_x) * sizeof(int);
    t.rec_off = b = up(b, 64);
    b += size_t(n_rec) * sizeof(long long);
    t.xs_off = b;
    b += size_t(n_x) * sizeof(long long);
    t.rec_w = b = up(b, 64);
    b += size_t(n_rec) * 8 * sizeof(float);
    t.bytes = up(b, 64);
    return t;
}

static int flow_tables(fd_handle *hd, int xb, int nbz, int nby, int nbx) {
    const int ns = int(hd->sources.size());
    const int n_x = ns > kFusedSources ? ns - kFusedSources : 0;
    if (hd->opt.storage != kF32 || (hd->n_rec == 0 && n_x == 0)) return FD_OK;
    if (hd->d_flow_tab && hd->flow_tab_gen == hd->gen && hd->flow_tab_xb == xb) return FD_OK;
    const long long regions = (long long)nbz * nby * nbx;
    auto region = [&](int x, int y, int z) {
        return (long long)(x / xb) * nby * nbz + (long long)(y / hd->tile_y) * nbz + z / hd->tile_z;
    };
    const FlowTables L = flow_table_layout(regions, hd->n_rec, n_x);
    std::vector<unsigned char> buf(L.bytes, 0);
    // counting sort of entries 0..count-1 by region: start[regions + 1], order[count]
    auto by_region = [&](const std::vector<long long> &reg, int *start, std::vector<int> &order) {
        for (long long g = 0; g <= regions; ++g) start[g] = 0;
        for (size_t i = 0; i < reg.size(); ++i) start[reg[i] + 1]++;
        for (long long g = 0; g < regions; ++g) start[g + 1] += start[g];
        std::vector<int> fill(start, start + regions);
        order.resize(reg.size());
        for (size_t i = 0; i < reg.size(); ++i) order[size_t(fill[size_t(reg[i])]++)] = int(i);
    };
    std::vector<int> order;
    if (hd->n_rec > 0) {
        std::vector<long long> reg(size_t(hd->n_rec));
        for (int r = 0; r < hd->n_rec; ++r) {
            const int *n = &hd->rec_node[size_t(r) * 3];
            reg[size_t(r)] = region(n[0], n[1], n[2]);
        }
        by_region(reg, reinterpret_cast<int *>(&buf[L.rec_start]), order);
        int *row = reinterpret_cast<int *>(&buf[L.rec_row]);
        long long *off = reinterpret_cast<long long *>(&buf[L.rec_off]);
        float *w = reinterpret_cast<float *>(&buf[L.rec_w]);
        for (size_t e = 0; e < order.size(); ++e) {
            const size_t r = size_t(order[e]);
            row[e] = int(r);
            off[e] = hd->rec_off_h[8 * r];  // corner c = 4 dx + 2 dy + dz: + dx plane + dy pz + dz
            for (int c = 0; c < 8; ++c) w[8 * e + size_t(c)] = hd->rec_w_h[8 * r + size_t(c)];
        }
    }
    if (n_x > 0) {
        std::vector<long long> reg(static_cast<size_t>(n_x));
        for (int i = 0; i < n_x; ++i) {
            const Source &q = hd->sources[size_t(i + kFusedSources)];
            reg[size_t(i)] = region(q.x, q.y, q.z);
        }
        by_region(reg, reinterpret_cast<int *>(&buf[L.xs_start]), order);
        int *idx = reinterpret_cast<int *>(&buf[L.xs_idx]);
        long long *off = reinterpret_cast<long long *>(&buf[L.xs_off]);
        for (size_t e = 0; e < order.size(); ++e) {
            const Source &q = hd->sources[size_t(order[e] + kFusedSources)];
            idx[e] = order[e] + kFusedSources;
            off[e] = (long long)q.x * hd->plane + (long long)q.y * hd->pz + q.z;
        }
    }
    if (hd->flow_tab_bytes < L.bytes) {
        dev_free(hd->d_flow_tab, hd->stream);
        hd->d_flow_tab = nullptr;
        hd->flow_tab_bytes = 0;
        if (dev_alloc(reinterpret_cast<void **>(&hd->d_flow_tab), L.bytes, hd->stream) != cudaSuccess) {
            cudaGetLastError();
            return fail(FD_ENOMEM, "cannot allocate the flow schedule's receiver and source tables");
        }
        hd->flow_tab_bytes = L.bytes;
    }
    if (reinterpret_cast<uintptr_t>(hd->d_flow_tab) % 64 != 0)
        return fail(FD_ECUDA, "flow tables not 64-byte aligned");
    FD_CUDA(cudaMemcpyAsync(hd->d_flow_tab, buf.data(), L.bytes, cudaMemcpyHostToDevice, hd->stream));
    FD_CUDA(cudaStreamSynchronize(hd->stream));  // the host table goes out of scope
    hd->gen++;  // graphs recorded with the old tables
    hd->flow_tab_gen = hd->gen;
    hd->flow_tab_xb = xb;
    return FD_OK;
}

// Flow launch arguments for nt steps from the handle's state with x-chunks of
// xb planes; *bytes: the zeroed prefix of the flow buffer (counter, abort, flags).
static int make_flow_args(fd_handle *hd, int nt, int xb, FlowArgs *f, size_t *bytes, int *ctas) {
    const int nbz = (hd->Nz + hd->tile_z - 1) / hd->tile_z, nby = (hd->Ny + hd->tile_y - 1) / hd->tile_y;
    const int nbx = (hd->Nx + xb - 1) / xb;
    const long long per_step = (long long)nbz * nby * nbx;
    // the work counter (an int) also counts one extra claim per CTA
    if (per_step * nt > INT32_MAX / 2) return fail(FD_EINVAL, "nt too large for one flow launch");
    *bytes = 16 + size_t(per_step) * sizeof(unsigned);
    if (hd->flow_bytes < *bytes) {
        dev_free(hd->flow_buf, hd->stream);
        hd->flow_buf = nullptr;
        hd->flow_bytes = 0;
        if (dev_alloc(&hd->flow_buf, *bytes, hd->stream) != cudaSuccess) {
            cudaGetLastError();
            return fail(FD_ENOMEM, "cannot allocate the flow schedule's flags");
        }
        hd->flow_bytes = *bytes;
        hd->gen++;  // graphs recorded with the old buffer
    }
    // the FP32 variant that samples receivers and adds extra sources per item
    const int ns = int(hd->sources.size()), n_x = ns > kFusedSources ? ns - kFusedSources : 0;
    const bool ex = hd->opt.storage == kF32 && (hd->n_rec > 0 || n_x > 0);
    int &flow_ctas = ex ? hd->flow_ctas_ex : hd->flow_ctas;
    if (flow_ctas == 0) {
        int dev = 0, sms = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        const int per_sm = tma_flow_ctas_per_sm(hd->r, hd->opt.form, hd->opt.storage, hd->tile_z, hd->tile_y,
                                                hd->rows, ex);
        if (per_sm <= 0 || sms <= 0) return fail(FD_ENOTSUP, "no flow kernel for this launch shape");
        flow_ctas = per_sm * sms;
    }
    f->maps[0] = hd->tmaps[0];
    f->maps[1] = hd->tmaps[1];
    f->a[0] = make_args(hd, hd->step, 0);
    f->a[1] = make_args(hd, hd->step, 1);
    f->a[0].x_block = f->a[1].x_block = xb;
    f->step0 = hd->step;
    f->nt = nt;
    f->cur0 = hd->cur;
    f->nbz = nbz;
    f->nby = nby;
    f->nbx = nbx;
    unsigned char *fb = static_cast<unsigned char *>(hd->flow_buf);
    f->counter = reinterpret_cast<int *>(fb);
    f->abort = reinterpret_cast<unsigned *>(fb + 4);
    f->amax = reinterpret_cast<unsigned *>(fb + 8);
    f->flags = reinterpret_cast<unsigned *>(fb + 16);
    f->a[0].n_rec = f->a[1].n_rec = 0;  // the flow kernel samples per item
    f->rec_start = f->rec_row = f->xs_start = f->xs_idx = nullptr;
    f->rec_off = f->xs_off = nullptr;
    f->rec_w = f->traces = nullptr;
    f->rec_stride = 0;
    f->rec_s0 = 0;
    f->xs_distinct = hd->extra_distinct ? 1 : 0;
    const int rc = flow_tables(hd, xb, nbz, nby, nbx);
    if (rc != FD_OK) return rc;
    if (ex) {
        const FlowTables L = flow_table_layout(per_step, hd->n_rec, n_x);
        unsigned char *t = hd->d_flow_tab;
        if (hd->n_rec > 0) {
            f->rec_start = reinterpret_cast<const int *>(t + L.rec_start);
            f->rec_row = reinterpret_cast<const int *>(t + L.rec_row);
            f->rec_off = reinterpret_cast<const long long *>(t + L.rec_off);
            f->rec_w = reinterpret_cast<const float *>(t + L.rec_w);
            f->traces = hd->d_traces;
            f->rec_stride = hd->rec_nt_max;
            f->rec_s0 = hd->rec_step0;
        }
        if (n_x > 0) {
            f->xs_start = reinterpret_cast<const int *>(t + L.xs_start);
            f->xs_idx = reinterpret_cast<const int *>(t + L.xs_idx);
            f->xs_off = reinterpret_cast<const long long *>(t + L.xs_off);
        }
    }
    *ctas = int(std::min<long long>(flow_ctas, per_step * nt));
    return FD_OK;
}

// One flow launch outside a graph (x_block tuning), timed by the handle's events.
static int flow_direct(fd_handle *hd, int nt, int xb, float *ms) {
    FlowArgs f;
    size_t bytes = 0;
    int ctas = 0;
    int rc = make_flow_args(hd, nt, xb, &f, &bytes, &ctas);
    if (rc != FD_OK) return rc;
    FD_CUDA(cudaEventRecord(hd->ev0, hd->stream));
    FD_CUDA(cudaMemsetAsync(hd->flow_buf, 0, bytes, hd->stream));
    FD_CUDA(launch_tma_flow(hd->r, hd->opt.form, hd->opt.storage, hd->tile_z, hd->tile_y, hd->rows, f, ctas,
                            check_enabled(hd), hd->stream));
    if (hd->opt.storage != kF32)
        FD_CUDA(launch_flow_finish_scales(hd->d_scales, int(((hd->step + nt) % 3 + 3) % 3), f.amax, hd->stream));
    FD_CUDA(sample_level(hd, hd->ubuf[hd->cur ^ (nt & 1)], hd->step + nt, hd->stream));
    FD_CUDA(cudaEventRecord(hd->ev1, hd->stream));
    FD_CUDA(cudaEventSynchronize(hd->ev1));
    FD_CUDA(cudaEventElapsedTime(ms, hd->ev0, hd->ev1));
    hd->step += nt;
    hd->cur ^= (nt & 1);
    return FD_OK;
}

// Launch shape and x_block of the single-step kernel, tuned on first use.
static int ensure_step_tuned(fd_handle *hd) {
    if (hd->kernel == kNaive || (hd->tile_y != 0 && hd->x_block != 0)) return FD_OK;
    int rc = autotune(hd);
    if (rc == FD_OK) rc = build_maps(hd);
    if (rc != FD_OK) {
        hd->tile_y = hd->x_block = 0;
        return rc;
    }
    hd->gen++;
    hd->flow_ctas = hd->flow_ctas_ex = 0;
    hd->flow_xb = 0;
    hd->flow_run_xb = 0;
    return FD_OK;
}

// nt steps of the single-step kernel, one launch per step, from the handle's graph.
static int run_steps(fd_handle *hd, int nt) {
    return replay_graph(hd, nt, false, [&](cudaStream_t st) {
        int cur = hd->cur;
        cudaError_t err = cudaSuccess;
        for (int i = 0; i < nt && err == cudaSuccess; ++i) {
            const StepArgs a = make_args(hd, hd->step + i, cur);
            err = enqueue_step(hd, a, st);
            cur ^= 1;
        }
        // the TMA kernel samples its input level: the last level of this forward is
        // sampled here (the next forward's first step samples it again, same values)
        if (err == cudaSuccess && hd->n_rec > 0 && hd->kernel == kTma)
            err = sample_level(hd, hd->ubuf[cur], hd->step + nt, st);
        return err;
    });
}

// nt steps in one flow launch with the handle's flow x_block, from its graph.
static int run_flow(fd_handle *hd, int nt) {
    FlowArgs f;
    size_t bytes = 0;
    int ctas = 0;
    int rc = make_flow_args(hd, nt, hd->flow_run_xb, &f, &bytes, &ctas);
    if (rc != FD_OK) return rc;
    const bool check = check_enabled(hd);
    return replay_graph(hd, nt, true, [&](cudaStream_t st) {
        cudaError_t e = cudaMemsetAsync(hd->flow_buf, 0, bytes, st);
        if (e == cudaSuccess)
            e = launch_tma_flow(hd->r, hd->opt.form, hd->opt.storage, hd->tile_z, hd->tile_y, hd->rows, f, ctas,
                                check, st);
        if (e == cudaSuccess && hd->opt.storage != kF32)
            e = launch_flow_finish_scales(hd->d_scales, int(((hd->step + nt) % 3 + 3) % 3), f.amax, st);
        // the items sample their input levels: the last level is sampled here
        if (e == cudaSuccess) e = sample_level(hd, hd->ubuf[hd->cur ^ (nt & 1)], hd->step + nt, st);
        return e;
    });
}

// nt per-step launches outside a graph (schedule tuning), timed by the handle's events.
static int steps_direct(fd_handle *hd, int nt, float *ms) {
    FD_CUDA(cudaEventRecord(hd->ev0, hd->stream));
    int cur = hd->cur;
    for (int i = 0; i < nt; ++i) {
        FD_CUDA(enqueue_step(hd, make_args(hd, hd->step + i, cur), hd->stream));
        cur ^= 1;
    }
    if (hd->kernel == kTma) FD_CUDA(sample_level(hd, hd->ubuf[cur], hd->step + nt, hd->stream));
    FD_CUDA(cudaEventRecord(hd->ev1, hd->stream));
    FD_CUDA(cudaEventSynchronize(hd->ev1));
    FD_CUDA(cudaEventElapsedTime(ms, hd->ev0, hd->ev1));
    hd->step += nt;
    hd->cur ^= (nt & 1);
    return FD_OK;
}

static bool flow_eligible(const fd_handle *hd) {
    const bool plain = hd->n_rec == 0 && int(hd->sources.size()) <= kFusedSources;
    return (hd->opt.storage == kF32 || (hd->opt.storage == kBF16 && plain)) && hd->kernel == kTma &&
           hd->opt.boundary == FD_BOUNDARY_ZERO && (hd->opt.x_block == 0 || hd->opt.x_block >= hd->r);
}

// Chooses the flow schedule's x_block and whether it beats per-step launches,
// timing the candidates on the first steps of this call (*nt is reduced by the
// steps they ran; every candidate computes the same bits). Cached per grid and
// launch shape for the process.
static int flow_prepare(fd_handle *hd, int *nt) {
    int rc = ensure_step_tuned(hd);
    if (rc != FD_OK) return rc;
    // the x_block the graphs use follows the chosen one
    auto use = [&](int xb) {
        if (xb != hd->flow_run_xb) {
            hd->flow_run_xb = xb;
            hd->gen++;
        }
        return FD_OK;
    };
    // receivers and extra sources change the balance of the two schedules: their
    // presence is part of the choice (made again when it changes)
    const int extras = (hd->n_rec > 0 ? 1 : 0) | (int(hd->sources.size()) > kFusedSources ? 2 : 0);
    if (hd->flow_xb != 0 && hd->flow_extras == extras) return use(hd->flow_xb);
    hd->flow_extras = extras;
    if (hd->opt.x_block > 0) {  // forced by the options
        hd->flow_xb = hd->opt.x_block;
        hd->flow_wins = true;
        return use(hd->flow_xb);
    }
    hd->flow_xb = 0;
    const auto key = std::make_tuple(hd->Nx, hd->Ny, hd->Nz, hd->r, hd->opt.form, hd->tile_z, hd->tile_y, extras);
    {
        std::lock_guard<std::mutex> lk(g_tune_mu);
        auto it = g_flow_cache.find(key);
        if (it != g_flow_cache.end()) {
            hd->flow_xb = it->second.first;
            hd->flow_wins = it->second.second;
            return use(hd->flow_xb);
        }
    }
    // shorter x-chunks balance better and keep more items in flight on small grids,
    // longer ones claim fewer items and re-read fewer queue planes
    constexpr int kTuneSteps = 8, kLongSteps = 24;
    std::vector<int> cand;
    for (int c : {8, 12, 16, 24, 32, 40, 48, 56, 64})
        if (c >= hd->r && c <= hd->Nx) cand.push_back(c);
    if (cand.empty()) cand.push_back(std::max(hd->r, 1));
    // warm-up + candidates, then the best length and the per-step launches each
    // timed afresh over kTuneSteps and kLongSteps
    const int needed = kTuneSteps * (int(cand.size()) + 1) + 2 * (kTuneSteps + kLongSteps);
    if (*nt < needed) {
        // too few steps to time: the usual best for this call, the timing left to a
        // later, longer call
        hd->flow_wins = true;
        return use(std::min(hd->Nx, std::max(40, hd->r)));
    }
    float ms = 0.0f, best = 1e30f, flow_short = 0.0f, flow_long = 0.0f, step_short = 0.0f, step_long = 0.0f;
    int best_xb = cand[0];
    rc = flow_direct(hd, kTuneSteps, cand[cand.size() / 2], &ms);  // warm-up
    for (int c : cand) {
        if (rc != FD_OK) break;
        rc = flow_direct(hd, kTuneSteps, c, &ms);
        if (rc == FD_OK && ms < best) {
            best = ms;
            best_xb = c;
        }
    }
    // schedule choice by differential timing: the cost of one more step, (t_long -
    // t_short) / (kLongSteps - kTuneSteps), for both schedules. A flow launch carries a
    // start-up and a last tail that a long run spreads out; the difference cancels them
    // (and the per-step launches' first-launch overhead) instead of a hand-set margin.
    // Both lengths are timed afresh: the candidates' minimum is biased low.
    if (rc == FD_OK) rc = flow_direct(hd, kTuneSteps, best_xb, &flow_short);
    if (rc == FD_OK) rc = flow_direct(hd, kLongSteps, best_xb, &flow_long);
    if (rc == FD_OK) rc = steps_direct(hd, kTuneSteps, &step_short);
    if (rc == FD_OK) rc = steps_direct(hd, kLongSteps, &step_long);
    if (rc != FD_OK) return rc;
    *nt -= needed;
    hd->flow_xb = best_xb;
    const float flow_per_step = (flow_long - flow_short) / float(kLongSteps - kTuneSteps);
    const float steps_per_step = (step_long - step_short) / float(kLongSteps - kTuneSteps);
    hd->flow_wins = flow_per_step <= steps_per_step;
    {
        std::lock_guard<std::mutex> lk(g_tune_mu);
        g_flow_cache[key] = std::make_pair(hd->flow_xb, hd->flow_wins);
    }
    return use(hd->flow_xb);
}

int fd_forward_flow(fd_handle *hd, int nt) {
    if (!hd) return fail(FD_EINVAL, "handle is NULL");
    if (hd->slab) return fail(FD_ENOTSUP, "a slab advances through fd_slab_step, with its halo exchange");
    if (nt < 0) return fail(FD_EINVAL, "nt must be >= 0");
    if (!hd->has_model) return fail(FD_ESTATE, "fd_forward_flow before fd_set_model");
    if (!flow_eligible(hd) && !(hd->opt.x_block > 0 && hd->opt.x_block < hd->r))
        return fail(FD_ENOTSUP,
                    "the flow schedule: FP32 storage (BF16 with <= %d sources and no receivers), TMA kernel, "
                    "zero boundary",
                    kFusedSources);
    // an item reads the queue planes and fronts of its x-neighbours only
    if (hd->opt.x_block > 0 && hd->opt.x_block < hd->r)
        return fail(FD_ENOTSUP, "the flow schedule needs x_block >= k/2");
    if (nt == 0) return FD_OK;
    int rc = flow_prepare(hd, &nt);
    if (rc != FD_OK || nt == 0) return rc;
    return run_flow(hd, nt);
}

int fd_read_wavefield(fd_handle *hd, float *out, int level) {
    if (!hd || !out) return fail(FD_EINVAL, "handle or out is NULL");
    if (level != 0 && level != 1) return fail(FD_EINVAL, "level must be 0 or 1");
    const int buf = level == 0 ? hd->cur : hd->cur ^ 1;
    const size_t row_bytes = size_t(hd->Nz) * sizeof(float);
    if (hd->opt.storage == kF32) {
        FD_CUDA(cudaMemcpy2DAsync(out, row_bytes, hd->ubuf[buf], size_t(hd->pz) * sizeof(float), row_bytes,
                                  size_t(hd->Nx) * hd->Ny, cudaMemcpyDeviceToHost, hd->stream));
    } else {
        const size_t n = size_t(hd->Nx) * hd->Ny * hd->Nz;
        if (!hd->d_unpack &&
            dev_alloc(reinterpret_cast<void **>(&hd->d_unpack), n * sizeof(float), hd->stream) != cudaSuccess)
            return fail(FD_ENOMEM, "cannot allocate the read-back buffer");
        FD_CUDA(unpack_to(hd, level, hd->d_unpack));
        FD_CUDA(cudaMemcpyAsync(out, hd->d_unpack, n * sizeof(float), cudaMemcpyDeviceToHost, hd->stream));
    }
    FD_CUDA(cudaStreamSynchronize(hd->stream));
    return check_enabled(hd) ? read_status(hd) : FD_OK;
}

int fd_read_wavefield_device(fd_handle *hd, float *d_out, int level) {
    if (!hd || !d_out) return fail(FD_EINVAL, "handle or out is NULL");
    if (level != 0 && level != 1) return fail(FD_EINVAL, "level must be 0 or 1");
    FD_CUDA(unpack_to(hd, level, d_out));
    return FD_OK;
}

int fd_set_stream(fd_handle *hd, void *cuda_stream) {
    if (!hd) return fail(FD_EINVAL, "handle is NULL");
    // work already queued on the old stream completes before the new one is used
    FD_CUDA(cudaStreamSynchronize(hd->stream));
    hd->stream = cuda_stream ? static_cast<cudaStream_t>(cuda_stream) : hd->own_stream;
    return FD_OK;
}

int fd_synchronize(fd_handle *hd) {
    if (!hd) return fail(FD_EINVAL, "handle is NULL");
    FD_CUDA(cudaStreamSynchronize(hd->stream));
    return check_enabled(hd) ? read_status(hd) : FD_OK;
}

int fd_status(fd_handle *hd) { return fd_synchronize(hd); }

int fd_load_state(fd_handle *hd, const float *u, const float *u_prev, long long step) {
    if (!hd || !u || !u_prev) return fail(FD_EINVAL, "handle or arrays are NULL");
    if (step < 0) return fail(FD_EINVAL, "step must be >= 0");
    const size_t n = size_t(hd->Nx) * hd->Ny * hd->Nz;
    const bool inc = hd->opt.storage != kF32;
    // levels as stored: FP32 (u^n, u^{n-1}); 16-bit (u^n, d^n = u^n - u^{n-1})
    std::vector<float> dvec;
    if (inc) dvec.resize(n);
    float amax[2] = {0.0f, 0.0f};
    for (size_t i = 0; i < n; ++i) {
        if (!std::isfinite(u[i]) || !std::isfinite(u_prev[i]))
            return fail(FD_EINVAL, "state value %zu is not finite", i);
        amax[0] = std::max(amax[0], std::fabs(u[i]));
        const float second = inc ? (dvec[i] = u[i] - u_prev[i]) : u_prev[i];
        amax[1] = std::max(amax[1], std::fabs(second));
    }
    const float *lv[2] = {u, inc ? dvec.data() : u_prev};
    void *dst[2] = {hd->ubuf[0], inc ? hd->dbuf : hd->ubuf[1]};
    float scale[2] = {1.0f, 1.0f};
    for (int l = 0; l < 2; ++l)
        if (inc && amax[l] > 0.0f) {
            int e;
            std::frexp(double(amax[l]) / 4096.0, &e);
            scale[l] = std::ldexp(1.0f, e);
        }
    float *tmp = nullptr;
    if (dev_alloc(reinterpret_cast<void **>(&tmp), n * sizeof(float), hd->stream) != cudaSuccess)
        return fail(FD_ENOMEM, "cannot allocate staging buffer");
    cudaError_t e = cudaSuccess;
    for (int l = 0; l < 2 && e == cudaSuccess; ++l) {
        e = cudaMemcpyAsync(tmp, lv[l], n * sizeof(float), cudaMemcpyHostToDevice, hd->stream);
        if (e == cudaSuccess)
            e = launch_pack_level(tmp, dst[l], hd->Nx, hd->Ny, hd->Nz, hd->pz, hd->opt.storage, 1.0f / scale[l],
                                  hd->stream);
        if (e == cudaSuccess) e = cudaStreamSynchronize(hd->stream);
    }
    unsigned bits[2];
    std::memcpy(bits, amax, sizeof bits);
    const int slot = int(((step % 3) + 3) % 3), next = int(((step + 1) % 3 + 3) % 3);
    if (e == cudaSuccess) e = launch_init_scales(hd->d_scales, hd->stream);
    if (e == cudaSuccess) e = launch_set_level_scale(hd->d_scales, slot, scale[0], bits[0], scale[1], bits[1], hd->stream);
    // the accumulators of the level the next step writes start at zero
    if (e == cudaSuccess) e = launch_set_level_scale(hd->d_scales, next, 1.0f, 0u, 1.0f, 0u, hd->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(hd->d_status, 0, sizeof(unsigned), hd->stream);
    dev_free(tmp, hd->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(hd->stream);
    if (e != cudaSuccess) return fail(FD_ECUDA, "loading state failed: %s", cudaGetErrorString(e));
    if (hd->n_rec > 0) {  // traces restart at the loaded step
        e = cudaMemsetAsync(hd->d_traces, 0, size_t(hd->n_rec) * hd->rec_nt_max * sizeof(float), hd->stream);
        if (e != cudaSuccess) return fail(FD_ECUDA, "loading state failed: %s", cudaGetErrorString(e));
    }
    hd->rec_step0 = step;
    hd->step = step;
    hd->cur = 0;
    return FD_OK;
}

int fd_reset(fd_handle *hd) {
    if (!hd) return fail(FD_EINVAL, "handle is NULL");
    const size_t ub = hd->n_pitched * elem_size(hd->opt.storage);
    FD_CUDA(cudaMemsetAsync(hd->ubuf[0], 0, ub, hd->stream));
    FD_CUDA(cudaMemsetAsync(hd->ubuf[1], 0, ub, hd->stream));
    if (hd->dbuf) FD_CUDA(cudaMemsetAsync(hd->dbuf, 0, ub, hd->stream));
    FD_CUDA(cudaMemsetAsync(hd->d_status, 0, sizeof(unsigned), hd->stream));
    FD_CUDA(launch_init_scales(hd->d_scales, hd->stream));
    if (hd->n_rec > 0)  // receivers keep their positions; their traces restart at step 0
        FD_CUDA(cudaMemsetAsync(hd->d_traces, 0, size_t(hd->n_rec) * hd->rec_nt_max * sizeof(float), hd->stream));
    hd->rec_step0 = 0;
    hd->step = 0;
    hd->cur = 0;
    return FD_OK;
}

int fd_get_step(fd_handle *hd, long long *step) {
    if (!hd || !step) return fail(FD_EINVAL, "NULL argument");
    *step = hd->step;
    return FD_OK;
}

int fd_get_dims(fd_handle *hd, int *Nx, int *Ny, int *Nz) {
    if (!hd || !Nx || !Ny || !Nz) return fail(FD_EINVAL, "NULL argument");
    *Nx = hd->Nx;
    *Ny = hd->Ny;
    *Nz = hd->Nz;
    return FD_OK;
}

int fd_get_config(fd_handle *hd, int *kernel, int *tile_z, int *tile_y, int *x_block) {
    if (!hd || !kernel || !tile_z || !tile_y || !x_block) return fail(FD_EINVAL, "NULL argument");
    *kernel = hd->kernel;
    *tile_z = hd->tile_z;
    *tile_y = hd->tile_y;
    *x_block = hd->x_block;
    return FD_OK;
}

int fd_get_schedule(fd_handle *hd, int *rows, int *schedule, int *flow_x_block) {
    if (!hd) return fail(FD_EINVAL, "handle is NULL");
    const bool tuned = hd->kernel == kNaive || (hd->tile_y != 0 && hd->x_block != 0);
    const bool two_step = hd->opt.kernel == kAuto && hd->kernel == kTma && hd->r == 1 &&
                          hd->opt.storage == kF32 && hd->opt.form == kFactored && hd->n_rec == 0 &&
                          int(hd->sources.size()) <= kFusedSources && !hd->slab;
    if (rows) *rows = tuned ? hd->rows : 0;
    // flow_run_xb: the x-chunk of the last flow call (also a short first call's)
    if (schedule)
        *schedule = !tuned ? 0
                    : two_step ? 2
                    : (hd->opt.kernel == kAuto && flow_eligible(hd) && hd->flow_wins && hd->flow_run_xb) ? 1
                                                                                                          : 0;
    if (flow_x_block) *flow_x_block = hd->flow_run_xb;
    return FD_OK;
}

int fd_last_forward_ms(fd_handle *hd, float *ms) {
    if (!hd || !ms) return fail(FD_EINVAL, "NULL argument");
    if (!hd->timed) return fail(FD_ESTATE, "no fd_forward timed yet");
    FD_CUDA(cudaEventSynchronize(hd->ev1));
    FD_CUDA(cudaEventElapsedTime(ms, hd->ev0, hd->ev1));
    return FD_OK;
}

// ---- slabs: one shot split along x ------------------------------------------

int fd_slab_create(int nx, int ny, int nz, int space_order, double h, double dt, int nbl, int x0, int x1,
                   const fd_options *opt, fd_handle **out) {
    if (x0 < 0 || x1 <= x0) {
        if (out) *out = nullptr;
        return fail(FD_EINVAL, "slab planes [%d, %d): need 0 <= x0 < x1", x0, x1);
    }
    return create_handle(nx, ny, nz, space_order, h, dt, nbl, opt, x0, x1, out);
}

int fd_slab_info(fd_handle *hd, int *x0, int *x1, int *ghost_lo, int *ghost_hi) {
    if (!hd) return fail(FD_EINVAL, "handle is NULL");
    if (x0) *x0 = hd->x_off + hd->x_lo;
    if (x1) *x1 = hd->x_off + hd->x_hi;
    if (ghost_lo) *ghost_lo = hd->ghost_lo;
    if (ghost_hi) *ghost_hi = hd->ghost_hi;
    return FD_OK;
}

int fd_slab_step(fd_handle *hd, int part) {
    if (!hd) return fail(FD_EINVAL, "handle is NULL");
    if (!hd->slab) return fail(FD_ENOTSUP, "fd_slab_step takes a slab (fd_slab_create)");
    if (part < FD_SLAB_BOUNDARY || part > FD_SLAB_ALL) return fail(FD_EINVAL, "part must be 1, 2 or 3");
    if (!hd->has_model) return fail(FD_ESTATE, "fd_slab_step before fd_set_model");
    int rc = ensure_step_tuned(hd);
    if (rc != FD_OK) return rc;
    const int r = hd->r, lo = hd->x_lo, hi = hd->x_hi;
    // [lo, b0) reads the low ghost planes, [b1, hi) the high ones, [b0, b1) neither
    const int b0 = hd->ghost_lo > 0 ? std::min(lo + r, hi) : lo;
    const int b1 = std::max(b0, hd->ghost_hi > 0 ? std::max(hi - r, lo) : hi);
    const StepArgs a = make_args(hd, hd->step, hd->cur);
    const TmaMaps &map = hd->tmaps[hd->cur];  // u^n in ubuf[cur]
    const bool check = check_enabled(hd);
    auto run = [&](int xa, int xb) -> cudaError_t {
        if (xb <= xa) return cudaSuccess;
        StepArgs b = a;
        b.x_lo = xa;
        b.x_hi = xb;
        return launch_tma_step(hd->r, hd->opt.form, kF32, hd->tile_z, hd->tile_y, hd->rows, map, b, check,
                               hd->stream);
    };
    if (part & FD_SLAB_BOUNDARY) {
        FD_CUDA(run(lo, b0));
        FD_CUDA(run(b1, hi));
    }
    if (part & FD_SLAB_INTERIOR) {
        FD_CUDA(run(b0, b1));
        hd->step += 1;
        hd->cur ^= 1;
    }
    return FD_OK;
}

int fd_slab_exchange_ptrs(fd_handle *hd, int level, void **send_lo, void **send_hi, void **recv_lo,
                          void **recv_hi, size_t *bytes) {
    if (!hd) return fail(FD_EINVAL, "handle is NULL");
    if (level != 0 && level != 1) return fail(FD_EINVAL, "level must be 0 or 1");
    char *buf = static_cast<char *>(hd->ubuf[level == 0 ? hd->cur : hd->cur ^ 1]);
    const size_t pb = size_t(hd->plane) * sizeof(float);
    if (send_lo) *send_lo = hd->ghost_lo > 0 ? buf + size_t(hd->x_lo) * pb : nullptr;
    if (send_hi) *send_hi = hd->ghost_hi > 0 ? buf + size_t(hd->x_hi - hd->r) * pb : nullptr;
    if (recv_lo) *recv_lo = hd->ghost_lo > 0 ? buf : nullptr;
    if (recv_hi) *recv_hi = hd->ghost_hi > 0 ? buf + size_t(hd->x_hi) * pb : nullptr;
    if (bytes) *bytes = size_t(hd->r) * pb;
    return FD_OK;
}

int fd_slab_exchange(fd_handle *from, fd_handle *to, int level, void *stream) {
    if (!from || !to) return fail(FD_EINVAL, "handle is NULL");
    if (!from->slab || !to->slab) return fail(FD_ENOTSUP, "fd_slab_exchange takes two slabs");
    if (level != 0 && level != 1) return fail(FD_EINVAL, "level must be 0 or 1");
    if (from->Ny != to->Ny || from->Nz != to->Nz || from->pz != to->pz || from->r != to->r ||
        from->Nx_glob != to->Nx_glob)
        return fail(FD_EINVAL, "the slabs belong to different shots");
    void *s_lo, *s_hi, *r_lo, *r_hi;
    size_t bytes = 0;
    fd_slab_exchange_ptrs(from, level, &s_lo, &s_hi, nullptr, nullptr, &bytes);
    fd_slab_exchange_ptrs(to, level, nullptr, nullptr, &r_lo, &r_hi, nullptr);
    const int from_end = from->x_off + from->x_hi, to_end = to->x_off + to->x_hi;
    const void *src = nullptr;
    void *dst = nullptr;
    if (from_end == to->x_off + to->x_lo && s_hi && r_lo) {
        src = s_hi;  // `to` is the right neighbour: its low ghosts
        dst = r_lo;
    } else if (to_end == from->x_off + from->x_lo && s_lo && r_hi) {
        src = s_lo;  // `to` is the left neighbour: its high ghosts
        dst = r_hi;
    } else {
        return fail(FD_EINVAL, "the slabs are not x-neighbours");
    }
    FD_CUDA(cudaMemcpyPeerAsync(dst, to->device, src, from->device, bytes, static_cast<cudaStream_t>(stream)));
    return FD_OK;
}

int fd_kernel_launches(long long *count) {
    if (!count) return fail(FD_EINVAL, "count is NULL");
    *count = kernel_launches();
    return FD_OK;
}

int fd_destroy(fd_handle *hd) {
    if (!hd) return FD_OK;
    if (hd->stream) cudaStreamSynchronize(hd->stream);
    release_handle(hd);
    return FD_OK;
}

}  // extern "C"

// ---------------------------------------------------------------------------
// Batches: many shots (different grids, same space order / h / storage / form)
// advanced together, one launch per time step over every shot's work items,
// replayed from a CUDA graph.
// ---------------------------------------------------------------------------

struct fd_batch {
    int k = 0, r = 0;
    double h = 0;
    fd_options opt{};
    int tile_z = 0, tile_y = 0;
    // x-chunk policy: every shot streams min(xb_policy, N_x) planes per CTA (0: whole
    // extents); tile and policy are timed on the first long forward unless forced
    int xb_policy = 0;
    bool tile_forced = false, tuned = false;
    cudaEvent_t tev0 = nullptr, tev1 = nullptr;
    std::vector<fd_handle *> slots;  // slot id -> shot (nullptr when free)
    BatchShot *d_shots = nullptr;
    size_t cap_shots = 0;
    int4 *d_items = nullptr;
    size_t cap_items = 0;
    int n_items = 0;
    std::vector<int> order;  // active slots in table order
    bool dirty = true;
    unsigned long long gen = 1;
    struct Graph {
        cudaGraphExec_t exec = nullptr;
        int nt = 0;
        unsigned long long gen = 0;
        bool flow = false;  // one persistent launch (else one launch per step)
    };
    std::vector<Graph> graphs;
    std::vector<int> seen_nt;              // chunk lengths launched once with this work list
    std::vector<cudaGraphExec_t> retired;  // replaced graphs, destroyed once the stream is idle
    std::vector<BatchShot> host_table;
    // flow schedule (FP32): one persistent launch per forward over every shot, chosen by
    // the autotuner when it times cheaper per step than the per-step launches. Per shot
    // (z tiles, y tiles, x-chunks, first work item); the work counter, abort word and one
    // flag per work item
    bool flow = false;
    bool flow_tuned = false;  // the schedule has been chosen (FP32), or there is no choice
    int4 *d_geo = nullptr;
    size_t cap_geo = 0;
    void *flow_buf = nullptr;
    size_t flow_cap = 0;
    int flow_ctas = 0;
    cudaStream_t own_stream = nullptr, stream = nullptr;
    cudaEvent_t join_ev = nullptr;
    // pinned staging for the argument table and the work list: uploads are
    // asynchronous, a buffer is rewritten only after its previous copy ran
    static constexpr int kStaging = 4;
    struct Staging {
        void *host = nullptr;
        size_t cap = 0;
        cudaEvent_t done = nullptr;
    };
    Staging staging[kStaging];
    int next_staging = 0;
};

namespace {

constexpr int kBatchXBlock = 96;

// Copy `bytes` from host memory to `dst` on the batch stream through the next
// pinned staging buffer (no host synchronisation unless that buffer's previous
// copy has not run yet).
int batch_stage_upload(fd_batch *b, void *dst, const void *src, size_t bytes) {
    if (bytes == 0) return FD_OK;
    fd_batch::Staging &sg = b->staging[b->next_staging];
    b->next_staging = (b->next_staging + 1) % fd_batch::kStaging;
    if (sg.done) FD_CUDA(cudaEventSynchronize(sg.done));
    if (sg.cap < bytes) {
        if (sg.host) cudaFreeHost(sg.host);
        sg.host = nullptr;
        sg.cap = 0;
        const size_t cap = std::max<size_t>(bytes, 4096) * 2;
        if (cudaMallocHost(&sg.host, cap) != cudaSuccess) return fail(FD_ENOMEM, "cannot allocate pinned staging");
        sg.cap = cap;
    }
    if (!sg.done) FD_CUDA(cudaEventCreateWithFlags(&sg.done, cudaEventDisableTiming));
    std::memcpy(sg.host, src, bytes);
    FD_CUDA(cudaMemcpyAsync(dst, sg.host, bytes, cudaMemcpyHostToDevice, b->stream));
    FD_CUDA(cudaEventRecord(sg.done, b->stream));
    return FD_OK;
}

// Grow a device array of the batch (stream-ordered: the old one is freed after
// the launches already queued that read it).
int batch_reserve(fd_batch *b, void **ptr, size_t *cap, size_t need, size_t elem) {
    if (need <= *cap) return FD_OK;
    const size_t old = *cap;  // grow geometrically: churn of added shots reallocates rarely
    dev_free(*ptr, b->stream);
    *ptr = nullptr;
    *cap = 0;
    const size_t n = std::max<size_t>(need, 2 * old);
    if (dev_alloc(ptr, n * elem, b->stream) != cudaSuccess) {
        cudaGetLastError();
        return fail(FD_ENOMEM, "cannot allocate a batch table");
    }
    *cap = n;
    return FD_OK;
}

void batch_destroy_retired(fd_batch *b) {
    for (auto e : b->retired) cudaGraphExecDestroy(e);
    b->retired.clear();
}

int batch_rebuild(fd_batch *b) {
    b->order.clear();
    std::vector<int4> items, geo;
    for (size_t s = 0; s < b->slots.size(); ++s) {
        fd_handle *hd = b->slots[s];
        if (!hd) continue;
        if (hd->stream != b->stream) {
            // a shot set up on its own stream joins the batch stream: the batch's next
            // launches wait for its set-up work (already finished in the usual case)
            FD_CUDA(cudaEventRecord(b->join_ev, hd->stream));
            FD_CUDA(cudaStreamWaitEvent(b->stream, b->join_ev, 0));
            hd->stream = b->stream;
        }
        const int idx = int(b->order.size());
        b->order.push_back(int(s));
        const int tz = (hd->Nz + b->tile_z - 1) / b->tile_z, ty = (hd->Ny + b->tile_y - 1) / b->tile_y;
        const int tx = (hd->Nx + hd->x_block - 1) / hd->x_block;
        geo.push_back(make_int4(tz, ty, tx, int(items.size())));
        for (int x = 0; x < tx; ++x)
            for (int y = 0; y < ty; ++y)
                for (int z = 0; z < tz; ++z) items.push_back(make_int4(idx, z, y, x));
    }
    int rc = batch_reserve(b, reinterpret_cast<void **>(&b->d_shots), &b->cap_shots, b->order.size(),
                           sizeof(BatchShot));
    if (rc == FD_OK)
        rc = batch_reserve(b, reinterpret_cast<void **>(&b->d_items), &b->cap_items, items.size(), sizeof(int4));
    if (rc == FD_OK) rc = batch_stage_upload(b, b->d_items, items.data(), items.size() * sizeof(int4));
    if (rc == FD_OK && b->opt.storage == kF32) {
        // the flow schedule's shot geometry and its counter, abort word and flags
        rc = batch_reserve(b, reinterpret_cast<void **>(&b->d_geo), &b->cap_geo, geo.size(), sizeof(int4));
        if (rc == FD_OK) rc = batch_stage_upload(b, b->d_geo, geo.data(), geo.size() * sizeof(int4));
        if (rc == FD_OK) rc = batch_reserve(b, &b->flow_buf, &b->flow_cap, 16 + items.size() * sizeof(unsigned), 1);
    }
    if (rc != FD_OK) return rc;
    b->n_items = int(items.size());
    // graphs of the old work list may still be queued: retire them, destroy them later
    for (auto &g : b->graphs)
        if (g.exec) b->retired.push_back(g.exec);
    b->graphs.clear();
    b->seen_nt.clear();
    if (b->retired.size() > 64) {
        FD_CUDA(cudaStreamSynchronize(b->stream));
        batch_destroy_retired(b);
    }
    b->dirty = false;
    b->gen++;
    return FD_OK;
}

int batch_upload_table(fd_batch *b) {
    b->host_table.resize(b->order.size());
    for (size_t i = 0; i < b->order.size(); ++i) {
        fd_handle *hd = b->slots[b->order[i]];
        BatchShot &t = b->host_table[i];
        for (int p = 0; p < 2; ++p) {
            t.args[p] = make_args(hd, hd->step, p);
            t.maps[p] = hd->tmaps[p];
        }
        t.cur0 = hd->cur;
        t.step0 = hd->step;
    }
    return batch_stage_upload(b, b->d_shots, b->host_table.data(), b->host_table.size() * sizeof(BatchShot));
}

// Every shot to the batch's launch shape: tile (tz, ty) and x-chunks of min(xb, N_x)
// planes (xb = 0: whole extents). The per-point arithmetic does not depend on
// either, so a shape change never changes a result.
int batch_apply_shape(fd_batch *b, int tz, int ty, int xb) {
    const bool tile_changed = tz != b->tile_z || ty != b->tile_y;
    b->tile_z = b->opt.tile_z = tz;
    b->tile_y = b->opt.tile_y = ty;
    b->xb_policy = xb;
    if (tile_changed) b->flow_ctas = 0;  // another kernel: its resident count is read again
    for (fd_handle *hd : b->slots) {
        if (!hd) continue;
        hd->x_block = xb > 0 ? std::min(xb, hd->Nx) : hd->Nx;
        hd->opt.x_block = hd->x_block;
        if (tile_changed) {
            hd->tile_z = hd->opt.tile_z = tz;
            hd->tile_y = hd->opt.tile_y = ty;
            hd->rows = 1;
            int rc = build_maps(hd);
            if (rc != FD_OK) return rc;
        }
    }
    b->dirty = true;
    return FD_OK;
}

// nt launches of the current work list, outside a graph, timed on the batch stream
// (the shots advance by nt steps).
int batch_timed_steps(fd_batch *b, int nt, float *ms) {
    int rc = batch_rebuild(b);
    if (rc == FD_OK) rc = batch_upload_table(b);
    if (rc != FD_OK) return rc;
    FD_CUDA(cudaEventRecord(b->tev0, b->stream));
    for (int i = 0; i < nt; ++i) {
        cudaError_t err = launch_tma_batch_step(b->r, b->opt.form, b->opt.storage, b->tile_z, b->tile_y, b->d_shots,
                                                b->d_items, b->n_items, i, b->stream);
        if (err != cudaSuccess) return fail(FD_ECUDA, "batch launch failed: %s", cudaGetErrorString(err));
    }
    FD_CUDA(cudaEventRecord(b->tev1, b->stream));
    FD_CUDA(cudaEventSynchronize(b->tev1));
    FD_CUDA(cudaEventElapsedTime(ms, b->tev0, b->tev1));
    for (int s : b->order) {
        fd_handle *hd = b->slots[s];
        hd->step += nt;
        hd->cur ^= (nt & 1);
    }
    return FD_OK;
}

// One persistent launch for nt steps of the current work list (FP32): the flags
// zeroed, then the launch, on stream st.
int batch_flow_enqueue(fd_batch *b, int nt, cudaStream_t st) {
    if (b->flow_ctas == 0) {
        int dev = 0, sms = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        const int per_sm = tma_batch_flow_ctas_per_sm(b->r, b->opt.form, b->tile_z, b->tile_y);
        if (per_sm <= 0 || sms <= 0) return fail(FD_ENOTSUP, "no batch flow kernel for this launch shape");
        b->flow_ctas = per_sm * sms;
    }
    if ((long long)b->n_items * nt > INT32_MAX / 2) return fail(FD_EINVAL, "nt too large for one batch flow launch");
    BatchFlowArgs f;
    unsigned char *fb = static_cast<unsigned char *>(b->flow_buf);
    f.shots = b->d_shots;
    f.items = b->d_items;
    f.geo = b->d_geo;
    f.n_items = b->n_items;
    f.nt = nt;
    f.counter = reinterpret_cast<int *>(fb);
    f.abort = reinterpret_cast<unsigned *>(fb + 4);
    f.flags = reinterpret_cast<unsigned *>(fb + 16);
    const size_t bytes = 16 + size_t(b->n_items) * sizeof(unsigned);
    const int ctas = int(std::min<long long>(b->flow_ctas, (long long)b->n_items * nt));
    cudaError_t err = cudaMemsetAsync(b->flow_buf, 0, bytes, st);
    if (err == cudaSuccess) err = launch_tma_batch_flow(b->r, b->opt.form, b->tile_z, b->tile_y, f, ctas, st);
    if (err != cudaSuccess) return fail(FD_ECUDA, "batch flow launch failed: %s", cudaGetErrorString(err));
    return FD_OK;
}

// One flow launch of nt steps outside a graph, timed on the batch stream (the shots
// advance by nt steps).
int batch_timed_flow(fd_batch *b, int nt, float *ms) {
    int rc = batch_rebuild(b);
    if (rc == FD_OK) rc = batch_upload_table(b);
    if (rc != FD_OK) return rc;
    FD_CUDA(cudaEventRecord(b->tev0, b->stream));
    rc = batch_flow_enqueue(b, nt, b->stream);
    if (rc != FD_OK) return rc;
    FD_CUDA(cudaEventRecord(b->tev1, b->stream));
    FD_CUDA(cudaEventSynchronize(b->tev1));
    FD_CUDA(cudaEventElapsedTime(ms, b->tev0, b->tev1));
    for (int s : b->order) {
        fd_handle *hd = b->slots[s];
        hd->step += nt;
        hd->cur ^= (nt & 1);
    }
    return FD_OK;
}

// Launch shapes timed by the batch autotuner: both tiles (unless forced) and
// x-chunk policies from short chunks (more CTAs, shorter queue warm-ups per
// chunk: neither) to whole extents.
constexpr int kBatchTuneSteps = 3;
constexpr int kBatchTuneXb[] = {32, 48, 64, 96, 128, 0};
constexpr int kBatchTuneMinShots = 4;
constexpr int kBatchLongSteps = 9;   // the long probes of the schedule choice
constexpr int kBatchFlowXb = 48;     // the flow's second x-chunk candidate

// Times every candidate shape on kBatchTuneSteps real steps of this forward (*nt is
// reduced by the steps they took) and keeps the fastest for the batch's lifetime.
// Runs once, on the first forward long enough with at least kBatchTuneMinShots shots.
// FP32 batches: whether one persistent launch per forward (the flow schedule) beats
// one launch per step on the tuned shape. The flow is timed at the tuned x-chunks and
// at kBatchFlowXb-plane chunks (shorter items balance a persistent launch better);
// then the cost of one more step of each schedule, (t_long - t_short) /
// (kBatchLongSteps - kBatchTuneSteps), decides (a flow launch's start-up and last
// tail cancel out). Runs once, on a forward with enough steps left (*nt is reduced
// by the steps it took; every probe is a real step of the batch).
int batch_flow_choice(fd_batch *b, int *nt) {
    const int n_fx = b->opt.x_block > 0 ? 1 : 2;
    const int needed = kBatchTuneSteps * n_fx + 2 * (kBatchTuneSteps + kBatchLongSteps);
    if (*nt < needed || int(b->order.size()) < kBatchTuneMinShots) return FD_OK;  // later, longer call
    const int tz = b->tile_z, ty = b->tile_y, xb0 = b->xb_policy;
    float ms = 0.0f, fbest = 1e30f;
    int fx = xb0;
    for (int xi = 0; xi < n_fx; ++xi) {
        const int xb = xi == 0 ? xb0 : kBatchFlowXb;
        int rc = batch_apply_shape(b, tz, ty, xb);
        if (rc == FD_OK) rc = batch_timed_flow(b, kBatchTuneSteps, &ms);
        if (rc != FD_OK) return rc;
        if (ms < fbest) {
            fbest = ms;
            fx = xb;
        }
    }
    float fs = 0.0f, fl = 0.0f, ss = 0.0f, sl = 0.0f;
    int rc = batch_apply_shape(b, tz, ty, fx);
    if (rc == FD_OK) rc = batch_timed_flow(b, kBatchTuneSteps, &fs);
    if (rc == FD_OK) rc = batch_timed_flow(b, kBatchLongSteps, &fl);
    if (rc == FD_OK) rc = batch_apply_shape(b, tz, ty, xb0);
    if (rc == FD_OK) rc = batch_timed_steps(b, kBatchTuneSteps, &ss);
    if (rc == FD_OK) rc = batch_timed_steps(b, kBatchLongSteps, &sl);
    if (rc != FD_OK) return rc;
    *nt -= needed;
    b->flow_tuned = true;
    b->flow = fl - fs <= sl - ss;
    return b->flow ? batch_apply_shape(b, tz, ty, fx) : FD_OK;
}

// Times every candidate shape on kBatchTuneSteps real steps of this forward (*nt is
// reduced by the steps they took) and keeps the fastest for the batch's lifetime.
// Runs once, on the first forward long enough with at least kBatchTuneMinShots shots;
// FP32 batches then choose their schedule (now if enough steps are left, else on a
// later forward).
int batch_autotune(fd_batch *b, int *nt) {
    int n_tiles = 0;
    int tiles[2][2];
    for (auto &t : kBatchTiles)
        if (!b->tile_forced || (t[0] == b->tile_z && t[1] == b->tile_y)) {
            tiles[n_tiles][0] = t[0];
            tiles[n_tiles][1] = t[1];
            ++n_tiles;
        }
    const int n_xb = b->opt.x_block > 0 ? 1 : int(sizeof(kBatchTuneXb) / sizeof(int));
    const int needed = kBatchTuneSteps * (n_tiles * n_xb + 1);
    if (*nt < needed || int(b->order.size()) < kBatchTuneMinShots) return FD_OK;  // later, longer call
    float best = 1e30f, ms = 0.0f;
    int best_t = 0, best_x = b->xb_policy;
    bool warmed = false;
    for (int ti = 0; ti < n_tiles; ++ti)
        for (int xi = 0; xi < n_xb; ++xi) {
            const int xb = b->opt.x_block > 0 ? b->opt.x_block : kBatchTuneXb[xi];
            int rc = batch_apply_shape(b, tiles[ti][0], tiles[ti][1], xb);
            if (rc == FD_OK && !warmed) {
                rc = batch_timed_steps(b, kBatchTuneSteps, &ms);  // the first launches run cold
                warmed = true;
            }
            if (rc == FD_OK) rc = batch_timed_steps(b, kBatchTuneSteps, &ms);
            if (rc != FD_OK) return rc;
            if (ms < best) {
                best = ms;
                best_t = ti;
                best_x = xb;
            }
        }
    *nt -= needed;
    b->tuned = true;
    int rc = batch_apply_shape(b, tiles[best_t][0], tiles[best_t][1], best_x);
    if (rc == FD_OK && !b->flow_tuned) rc = batch_flow_choice(b, nt);
    return rc;
}

fd_handle *batch_shot(fd_batch *b, int slot) {
    if (!b || slot < 0 || size_t(slot) >= b->slots.size()) return nullptr;
    return b->slots[slot];
}

// schedule: -1 the batch's own (autotuned), 1 one persistent launch
int batch_forward(fd_batch *b, int nt, int schedule) {
    if (!b) return fail(FD_EINVAL, "batch is NULL");
    if (nt < 0) return fail(FD_EINVAL, "nt must be >= 0");
    if (b->dirty) {
        int rc = batch_rebuild(b);
        if (rc != FD_OK) return rc;
    }
    if (nt == 0 || b->order.empty()) return FD_OK;
    if (!b->tuned || !b->flow_tuned) {
        int rc = b->tuned ? batch_flow_choice(b, &nt) : batch_autotune(b, &nt);
        if (rc != FD_OK) return rc;
        if (b->dirty) {
            rc = batch_rebuild(b);
            if (rc != FD_OK) return rc;
        }
        if (nt == 0) return FD_OK;
    }
    int rc = batch_upload_table(b);
    if (rc != FD_OK) return rc;
    const bool flow = b->opt.storage == kF32 && (schedule == 1 || b->flow);
    fd_batch::Graph *g = nullptr;
    for (auto &e : b->graphs)
        if (e.nt == nt && e.gen == b->gen && e.flow == flow) g = &e;
    // a chunk length seen for the first time with this work list is launched
    // directly (capturing a graph costs more than one replay saves); the second
    // time it is captured and replayed from then on
    const bool first = std::find(b->seen_nt.begin(), b->seen_nt.end(), nt) == b->seen_nt.end();
    if (!g && first) {
        b->seen_nt.push_back(nt);
        if (flow) {
            rc = batch_flow_enqueue(b, nt, b->stream);
            if (rc != FD_OK) return rc;
        }
        for (int i = 0; i < nt && !flow; ++i) {
            cudaError_t err = launch_tma_batch_step(b->r, b->opt.form, b->opt.storage, b->tile_z, b->tile_y,
                                                    b->d_shots, b->d_items, b->n_items, i, b->stream);
            if (err != cudaSuccess) return fail(FD_ECUDA, "batch launch failed: %s", cudaGetErrorString(err));
        }
    } else if (!g) {
        cudaGraph_t graph = nullptr;
        FD_CUDA(cudaStreamBeginCapture(b->stream, cudaStreamCaptureModeThreadLocal));
        cudaError_t err = cudaSuccess;
        if (flow && batch_flow_enqueue(b, nt, b->stream) != FD_OK) err = cudaErrorLaunchFailure;
        for (int i = 0; i < nt && err == cudaSuccess && !flow; ++i)
            err = launch_tma_batch_step(b->r, b->opt.form, b->opt.storage, b->tile_z, b->tile_y, b->d_shots,
                                        b->d_items, b->n_items, i, b->stream);
        cudaError_t cap = cudaStreamEndCapture(b->stream, &graph);
        if (err != cudaSuccess || cap != cudaSuccess) {
            if (graph) cudaGraphDestroy(graph);
            return fail(FD_ECUDA, "batch graph capture failed: %s", cudaGetErrorString(err != cudaSuccess ? err : cap));
        }
        cudaGraphExec_t exec = nullptr;
        cudaError_t ie = cudaGraphInstantiate(&exec, graph, 0);
        cudaGraphDestroy(graph);
        if (ie != cudaSuccess) return fail(FD_ECUDA, "cudaGraphInstantiate failed: %s", cudaGetErrorString(ie));
        if (b->graphs.size() >= 8) {
            b->retired.push_back(b->graphs.front().exec);  // may still be queued
            b->graphs.erase(b->graphs.begin());
        }
        b->graphs.push_back({exec, nt, b->gen, flow});
        g = &b->graphs.back();
    }
    if (g) {
        FD_CUDA(cudaGraphLaunch(g->exec, b->stream));
        count_replay(g->flow ? 1 : nt);  // one batch kernel per step, or one persistent launch
    }
    for (int s : b->order) {
        fd_handle *hd = b->slots[s];
        hd->step += nt;
        hd->cur ^= (nt & 1);
    }
    return FD_OK;
}

}  // namespace

extern "C" {

int fd_shot_device_bytes(int nx, int ny, int nz, int nbl, int storage, long long *out) {
    if (!out || nx < 1 || ny < 1 || nz < 1 || nbl < 0 || storage < 0 || storage > 2)
        return fail(FD_EINVAL, "bad extents or storage");
    const long long Nx = nx + 2LL * nbl, Ny = ny + 2LL * nbl, Nz = nz + 2LL * nbl;
    const long long pz = (Nz + 63) / 64 * 64;
    const long long n = Nx * Ny * pz;
    const int fields = storage == kF32 ? 2 : 3;  // 16-bit keeps u in two buffers plus the increment
    *out = fields * n * (long long)elem_size(storage) + 2 * n * 4 + (1 << 16);
    return FD_OK;
}

int fd_batch_create(int space_order, double h, const fd_options *opt_in, fd_batch **out) {
    if (!out) return fail(FD_EINVAL, "out is NULL");
    *out = nullptr;
    if (space_order < 2 || space_order > 2 * kMaxBatchRadius || space_order % 2)
        return fail(FD_EINVAL, "batches take space orders even in [2, 16], got %d", space_order);
    if (!(h > 0) || !std::isfinite(h)) return fail(FD_EINVAL, "h must be positive and finite");
    fd_options opt;
    fd_options_default(&opt);
    if (opt_in) opt = *opt_in;
    if (opt.storage < 0 || opt.storage > 2 || opt.form < 0 || opt.form > 1)
        return fail(FD_ENOTSUP, "unknown storage/form option");
    if (opt.storage != kF32 && opt.form != kFactored)
        return fail(FD_ENOTSUP, "batches with 16-bit storage use the factored form");
    if (opt.boundary != FD_BOUNDARY_ZERO) return fail(FD_ENOTSUP, "batches use the zero boundary");
    int tz = opt.tile_z, ty = opt.tile_y;
    if (tz == 0 && ty == 0) {
        tz = kBatchTiles[0][0];
        ty = kBatchTiles[0][1];
    }
    bool ok = false;
    for (auto &t : kBatchTiles) ok |= (t[0] == tz && t[1] == ty);
    if (!ok) return fail(FD_ENOTSUP, "batch tile must be 32x16 or 64x8");
    if (opt.rows > 1) return fail(FD_ENOTSUP, "batches run one row per thread");
    fd_batch *b = new fd_batch();
    b->tile_forced = opt.tile_z != 0 || opt.tile_y != 0;
    b->xb_policy = opt.x_block > 0 ? opt.x_block : kBatchXBlock;
    b->tuned = opt.x_block > 0 && b->tile_forced;  // no shape left to time
    // the schedule is timed for FP32 batches whose x-chunks the flow can take
    b->flow_tuned = opt.storage != kF32 || (opt.x_block > 0 && opt.x_block < space_order / 2) ||
                    opt.kernel == kTma;  // kernel TMA: one launch per step, pinned
    b->k = space_order;
    b->r = space_order / 2;
    b->h = h;
    b->opt = opt;
    b->opt.kernel = kTma;
    b->opt.tile_z = tz;
    b->opt.tile_y = ty;
    b->opt.check_finite = 1;
    b->tile_z = tz;
    b->tile_y = ty;
    if (cudaStreamCreateWithFlags(&b->own_stream, cudaStreamNonBlocking) != cudaSuccess ||
        cudaEventCreateWithFlags(&b->join_ev, cudaEventDisableTiming) != cudaSuccess ||
        cudaEventCreate(&b->tev0) != cudaSuccess || cudaEventCreate(&b->tev1) != cudaSuccess) {
        if (b->own_stream) cudaStreamDestroy(b->own_stream);
        delete b;
        return fail(FD_ECUDA, "cudaStreamCreate failed");
    }
    b->stream = b->own_stream;
    *out = b;
    return FD_OK;
}

int fd_batch_add(fd_batch *b, int nx, int ny, int nz, int nbl, double dt, const float *m, const float *eta,
                 int *slot) {
    if (!b || !m || !slot) return fail(FD_EINVAL, "batch, m or slot is NULL");
    // tile fixed by the batch; x_block forced, else long x-runs: a batch has work items to
    // spare, so it trades CTA count for fewer queue warm-ups (measured best near 96 planes)
    fd_options opt = b->opt;
    opt.x_block = b->xb_policy > 0 ? std::min(b->xb_policy, nx + 2 * nbl) : nx + 2 * nbl;
    fd_handle *hd = nullptr;
    int rc = fd_acoustic_create_ex(nx, ny, nz, b->k, b->h, dt, nbl, &opt, &hd);
    if (rc != FD_OK) return rc;
    // set-up (model upload and checks, sources) runs on the shot's own stream, so it
    // neither waits for nor stalls the batch's launches; the shot moves to the batch
    // stream when the next forward rebuilds the work list
    rc = fd_set_model(hd, m, eta);
    if (rc == FD_OK) rc = autotune(hd);
    if (rc == FD_OK) rc = build_maps(hd);
    if (rc != FD_OK) {
        std::string msg = g_last_error;
        fd_destroy(hd);
        return fail(rc, "%s", msg.c_str());
    }
    int s = -1;
    for (size_t i = 0; i < b->slots.size(); ++i)
        if (!b->slots[i]) {
            s = int(i);
            break;
        }
    if (s < 0) {
        s = int(b->slots.size());
        b->slots.push_back(nullptr);
    }
    b->slots[s] = hd;
    b->dirty = true;
    *slot = s;
    return FD_OK;
}

int fd_batch_inject(fd_batch *b, int slot, int ix, int iy, int iz, const float *wavelet, int nt) {
    fd_handle *hd = batch_shot(b, slot);
    if (!hd) return fail(FD_EINVAL, "no shot in slot %d", slot);
    if (int(hd->sources.size()) >= kFusedSources)
        return fail(FD_ENOTSUP, "a batched shot holds at most %d sources", kFusedSources);
    int rc = fd_inject(hd, ix, iy, iz, wavelet, nt);
    if (rc == FD_OK) b->dirty = true;  // argument tables carry the sources
    return rc;
}

int fd_batch_remove(fd_batch *b, int slot) {
    fd_handle *hd = batch_shot(b, slot);
    if (!hd) return fail(FD_EINVAL, "no shot in slot %d", slot);
    b->slots[slot] = nullptr;
    b->dirty = true;
    // its fields are freed in stream order, after the launches already queued that use them
    release_handle(hd);
    return FD_OK;
}

int fd_batch_forward(fd_batch *b, int nt) { return batch_forward(b, nt, -1); }

int fd_batch_forward_flow(fd_batch *b, int nt) {
    if (b && b->opt.storage != kF32) return fail(FD_ENOTSUP, "the batch flow schedule stores FP32");
    // an item reads the queue planes and fronts of its x-neighbour chunks only
    if (b && b->xb_policy > 0 && b->xb_policy < b->r)
        return fail(FD_ENOTSUP, "the batch flow schedule needs x_block >= k/2");
    return batch_forward(b, nt, 1);
}

int fd_batch_schedule(fd_batch *b, int *flow) {
    if (!b || !flow) return fail(FD_EINVAL, "batch or flow is NULL");
    *flow = b->flow ? 1 : 0;
    return FD_OK;
}

int fd_batch_read(fd_batch *b, int slot, float *out, int level) {
    fd_handle *hd = batch_shot(b, slot);
    if (!hd) return fail(FD_EINVAL, "no shot in slot %d", slot);
    return fd_read_wavefield(hd, out, level);
}

int fd_batch_read_device(fd_batch *b, int slot, float *d_out, int level) {
    fd_handle *hd = batch_shot(b, slot);
    if (!hd) return fail(FD_EINVAL, "no shot in slot %d", slot);
    return fd_read_wavefield_device(hd, d_out, level);
}

int fd_batch_shot_step(fd_batch *b, int slot, long long *step) {
    fd_handle *hd = batch_shot(b, slot);
    if (!hd) return fail(FD_EINVAL, "no shot in slot %d", slot);
    return fd_get_step(hd, step);
}

int fd_batch_shot_status(fd_batch *b, int slot) {
    fd_handle *hd = batch_shot(b, slot);
    if (!hd) return fail(FD_EINVAL, "no shot in slot %d", slot);
    return fd_status(hd);
}

int fd_batch_size(fd_batch *b, int *active, int *work_items) {
    if (!b || !active || !work_items) return fail(FD_EINVAL, "NULL argument");
    int n = 0;
    for (auto *hd : b->slots) n += hd != nullptr;
    *active = n;
    *work_items = b->dirty ? -1 : b->n_items;
    return FD_OK;
}

int fd_batch_reset(fd_batch *b) {
    if (!b) return fail(FD_EINVAL, "batch is NULL");
    for (auto *hd : b->slots)
        if (hd) {
            int rc = fd_reset(hd);
            if (rc != FD_OK) return rc;
        }
    return FD_OK;
}

int fd_batch_set_stream(fd_batch *b, void *cuda_stream) {
    if (!b) return fail(FD_EINVAL, "batch is NULL");
    FD_CUDA(cudaStreamSynchronize(b->stream));
    b->stream = cuda_stream ? static_cast<cudaStream_t>(cuda_stream) : b->own_stream;
    for (auto *hd : b->slots)
        if (hd) hd->stream = b->stream;
    return FD_OK;
}

int fd_batch_synchronize(fd_batch *b) {
    if (!b) return fail(FD_EINVAL, "batch is NULL");
    FD_CUDA(cudaStreamSynchronize(b->stream));
    batch_destroy_retired(b);
    return FD_OK;
}

int fd_batch_destroy(fd_batch *b) {
    if (!b) return FD_OK;
    cudaStreamSynchronize(b->stream);
    for (auto *hd : b->slots)
        if (hd) {
            cudaStreamSynchronize(hd->stream);
            release_handle(hd);
        }
    for (auto &g : b->graphs)
        if (g.exec) cudaGraphExecDestroy(g.exec);
    batch_destroy_retired(b);
    dev_free(b->d_shots, b->stream);
    dev_free(b->d_items, b->stream);
    dev_free(b->d_geo, b->stream);
    dev_free(b->flow_buf, b->stream);
    cudaStreamSynchronize(b->stream);
    for (auto &sg : b->staging) {
        if (sg.done) cudaEventDestroy(sg.done);
        if (sg.host) cudaFreeHost(sg.host);
    }
    if (b->join_ev) cudaEventDestroy(b->join_ev);
    if (b->tev0) cudaEventDestroy(b->tev0);
    if (b->tev1) cudaEventDestroy(b->tev1);
    if (b->own_stream) cudaStreamDestroy(b->own_stream);
    delete b;
    return FD_OK;
}

int fd_batch_get_config(fd_batch *b, int *tile_z, int *tile_y, int *x_block, int *tuned) {
    if (!b) return fail(FD_EINVAL, "batch is NULL");
    if (tile_z) *tile_z = b->tile_z;
    if (tile_y) *tile_y = b->tile_y;
    if (x_block) *x_block = b->xb_policy;
    if (tuned) *tuned = b->tuned ? 1 : 0;
    return FD_OK;
}

}  // extern "C"
