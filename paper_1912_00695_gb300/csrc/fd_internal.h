// Internal declarations shared by the host runtime and the kernel translation
// units. Not part of the public ABI (include/fd_acoustic.h is).
#pragma once

#include <cstddef>
#include <cstdint>

#include <cuda.h>
#include <cuda_runtime.h>

namespace fdgb {

constexpr int kMaxRadius = 12;      // space order 24
constexpr int kMaxBatchRadius = 8;  // batches: space order 16
constexpr int kMaxRadiusHost = 12;  // host weight generator reaches space order 24
constexpr int kFusedSources = 4;    // sources injected inside the step kernel (more: one extra kernel)
// Epilogue modes of the FP32 factored TMA step (the FWI gradient's two passes):
// kModeStep the plain step; kModeForwardD also stores the second time
// difference D^n = u^{n+1} - 2u^n + u^{n-1} (this step's fused sources
// included) into StepArgs::hist; kModeAdjointGrad (the adjoint field w^k
// computed over w^{k+2} from w^{k+1}) accumulates grad -= w^k * D^{k-1}, D
// read from StepArgs::hist.
constexpr int kModeStep = 0, kModeForwardD = 1, kModeAdjointGrad = 2;
// TMA kernel: registers capped for 16 resident warps per SM (the kernel is
// latency-bound: occupancy is worth more than the few spill slots this costs
// at R = 8).
constexpr int kTmaWarpsPerSM = 16;
// above radius 8 the register queue needs more than 128 registers per thread:
// 8 warps per SM
// Two y rows per thread double the x queues: 8 warps per SM as well.
constexpr int tma_warps_per_sm(int r, int rows = 1) { return (r > 8 || rows > 1) ? 8 : kTmaWarpsPerSM; }
constexpr int kTileZ = 32;          // streaming tile width along z (one warp)
constexpr int kMaxDim = 65535;  // keeps every launch grid dimension within limits

enum Storage : int { kF32 = 0, kBF16 = 1, kF16 = 2 };
enum Form : int { kFactored = 0, kExpanded = 1 };
enum KernelKind : int { kAuto = 0, kStream = 1, kNaive = 2, kTma = 3 };

// Device status word bits (written by kernels, read by the host).
constexpr unsigned kStatusNonFinite = 1u;
constexpr unsigned kStatusTimeout = 2u;  // a bounded device-side wait gave up

// Per-level scale bookkeeping for 16-bit storage, which keeps u^n and the
// increment d^n = u^n - u^{n-1} (value = stored * scale). Three rotating slots,
// indexed by global step modulo 3: slot (n % 3) holds the scales of u^n and d^n
// and the max |u^n|, |d^n| accumulated while they were written.
struct LevelScales {
    float scale[3];          // u^n
    float dscale[3];         // d^n
    unsigned amax_bits[3];   // max |u| as float bits (non-negative floats order as uints)
    unsigned damax_bits[3];  // max |d|
};

// Arguments of one time step of one shot. Passed by value (kernel parameter
// space) for the single-shot kernels and stored in device memory for batches.
struct StepArgs {
    const void *u;      // u^n, storage type, pitched [Nx][Ny][pz]
    void *up;           // FP32: u^{n-1} on entry, overwritten by u^{n+1};
                        // 16-bit: the increment d^n on entry, overwritten by d^{n+1}
    void *un;           // 16-bit: receives u^{n+1} (the buffer that held u^{n-1}); FP32: null
    const float *f1;    // factored: w = dt^2/(m + dt/2 eta); expanded: m
    const float *f2;    // factored: g = (dt/2 eta)/(m + dt/2 eta); expanded: eta
    int Nx, Ny, Nz;     // computational domain
    int pz;             // row pitch in elements (multiple of 32)
    long long plane;    // elements per x-plane = Ny * pz
    int x_block;        // planes per CTA (streaming kernel)
    int x_lo, x_hi;     // planes the TMA step kernel updates: [x_lo, x_hi) (a slab's own
                        // planes; [0, Nx) otherwise). Planes outside are read, not written.
    // box where f2 == 0 (damping absent): [bx0,bx1) x [by0,by1) x [bz0,bz1)
    int bx0, bx1, by0, by1, bz0, bz1;
    float coef[kMaxRadius + 1];  // factored: c_j/h^2; expanded: c_j dt^2/h^2 (j >= 1;
                                 // the centre enters as -u_c in every tap)
    float half_dt;               // dt/2 (expanded form)
    float dt2;                   // dt^2 (expanded form: source weight dt^2 / r0)
    // fused sources: domain node and wavelet row
    int ns;
    int sx[kFusedSources], sy[kFusedSources], sz[kFusedSources];
    const float *wavelet;  // ns rows of ld samples
    int ld;
    long long step;        // global step n (u^n -> u^{n+1})
    // status / 16-bit scales (may be null for FP32 without finite check)
    unsigned *status;
    LevelScales *scales;
    float src_bound;       // max_s |w_s q_s| bound used by 16-bit scale selection
    // receivers (single-shot TMA kernel): the step samples its input level u^n
    // into traces[r * rec_stride + rec_sample]; rec_sample < 0: no sample
    const long long *rec_off;  // 8 pitched offsets per receiver
    const float *rec_w;        // 8 trilinear weights per receiver
    float *traces;
    int n_rec, rec_stride, rec_sample;
    // FWI gradient passes: this step's slot of the second-time-difference
    // history (forward: written; adjoint: read) and the gradient (adjoint)
    float *hist;
    float *grad;
    int hist_slot;  // adjoint pass: the history level D^{k-1} sits at
};

// Host numerics (fd_numerics.cpp)
bool fornberg_second_derivative(int space_order, double *c);
double stability_limit(int space_order, double h, double vmax);
void default_damping(const float *m, float *eta, int Nx, int Ny, int Nz, int nbl, double h,
                     double vmax);

// Kernel launchers (fd_kernels_r*.cu). Return cudaSuccess or the launch error.
cudaError_t launch_stream_step(int radius, int form, int storage, int tile_y, const StepArgs &a,
                               bool check, cudaStream_t s);
cudaError_t launch_naive_step(int radius, int form, int storage, const StepArgs &a, bool check,
                              cudaStream_t s);
int stream_grid_x_chunks(int Nx, int x_block);
// Tensor maps of one step of the TMA kernel: u^n with the halo box (copied into
// the shared ring), and the point boxes (tile without halo) of u^n, u^{n-1},
// w (m) and g (eta), used only for L2 prefetches.
struct TmaMaps {
    CUtensorMap u_halo;
    CUtensorMap u_pt;
    CUtensorMap up_pt;
    CUtensorMap f1_pt;
    CUtensorMap f2_pt;
};

// The FWI gradient's adjoint pass reads these through the ring too.
struct GradMaps {
    CUtensorMap hist;  // 4-D: the second-time-difference history [levels][Nx][Ny][pz]
    CUtensorMap grad;  // 3-D: the gradient
};

// One shot of a batch as the batched kernel sees it (device memory): the step
// arguments and tensor maps for both buffer parities (index p: u^n in buffer
// p), the parity and global step of u^n at the start of the launch sequence.
struct BatchShot {
    StepArgs args[2];
    TmaMaps maps[2];
    int cur0;
    long long step0;
};

// Tile shapes of the batched kernel (every storage and form).
constexpr int kBatchTiles[2][2] = {{32, 16}, {64, 8}};

// Batched TMA kernel (fd_tma.cuh): one CTA per work item (shot, tile_z index,
// tile_y index, x chunk); `offset` is the step's index within the launch sequence.
cudaError_t launch_tma_batch_step(int radius, int form, int storage, int tile_z, int tile_y,
                                  const BatchShot *shots, const int4 *items, int n_items, int offset,
                                  cudaStream_t s);

// TMA-fed kernel (fd_tma.cuh): FP32 storage in tiles (tile_z, tile_y) of {(32,32), (64,16),
// (128,8), (32,16), (64,8)} and both forms; 16-bit storage in (32,16) and (64,8), factored
// form. The halo box of `maps.u_halo` is (box_w, box_h, 1) from tma_box (false: no such
// configuration).
// `rows`: y rows per thread (1, or 2 in the shapes of FDGB_TMA_CONFIGS2; the
// tile's tile_y counts the rows of all threads).
cudaError_t launch_tma_step(int radius, int form, int storage, int tile_z, int tile_y, int rows,
                            const TmaMaps &maps, const StepArgs &a, bool check, cudaStream_t s);
bool tma_box(int radius, int form, int storage, int tile_z, int tile_y, int rows, int *box_w, int *box_h,
             int *rz);

// Utility kernels (fd_kernels_util.cu)
cudaError_t launch_inject_extra(const StepArgs &a, const int *sx, const int *sy, const int *sz,
                                int first, int count, int storage, int expanded, bool distinct, cudaStream_t s,
                                float *hist = nullptr);
cudaError_t launch_residual(const float *syn, float *obs_to_res, size_t n, cudaStream_t s);
cudaError_t launch_adjoint_inject(float *w, float *grad, const float *dhist, const float *f1,
                                  const long long *node_off, const int *row, const int *rec_idx, const float *rec_w,
                                  const float *resid, int nt, int t, float inv_dt2, int n_nodes, cudaStream_t s);
// Two steps per launch (FP32 factored, radius 1-2): u^{n+1} into out1, u^{n+2} into out2.
cudaError_t launch_tma2_step(int radius, const TmaMaps &map, const StepArgs &a, float *out1, float *out2, bool check,
                             cudaStream_t s);
bool tma2_geometry(int radius, int *tz, int *ty, int *box_w, int *box_h, int *ez, int *ey);
cudaError_t launch_tma_grad_step(int radius, int mode, const TmaMaps &map, const GradMaps &gm, const StepArgs &a,
                                 bool check, cudaStream_t s);
cudaError_t launch_sample_receivers(const void *u, int storage, const LevelScales *scales, int slot,
                                    const long long *off, const float *w, int n, float *out, int stride,
                                    cudaStream_t s);
cudaError_t launch_unpack_level(const void *src, float *dst, int Nx, int Ny, int Nz, int pz,
                                int storage, const LevelScales *scales, int slot,
                                cudaStream_t s);
cudaError_t launch_init_scales(LevelScales *scales, cudaStream_t s);

// Model set-up on the device (fd_set_model*): validation and min(m) in one pass,
// the default damping profile, and the factored form's derived coefficients.
struct ModelCheck {
    unsigned bad_m;                 // some m is not positive finite
    unsigned bad_eta;               // some eta is negative or not finite
    unsigned min_m_bits;            // min m as float bits (positive floats order as uints)
    unsigned eta_interior_nonzero;  // eta != 0 somewhere inside the interior box
};
// x_off: global plane of local plane 0 and Nx_glob the global extent (a slab's
// window onto the domain; 0 and Nx otherwise), for the interior box test.
cudaError_t launch_model_check(const float *m, const float *eta, int Nx, int Ny, int Nz, int pz, int nbl,
                               int x_off, int Nx_glob, ModelCheck *out, cudaStream_t s);
cudaError_t launch_default_damping(const float *m, float *eta, int Nx, int Ny, int Nz, int pz, int nbl,
                                   float dmax, cudaStream_t s);
cudaError_t launch_prepare_factored(float *f1, float *f2, long long n_pitched, float half_dt, float dt2,
                                    cudaStream_t s);
cudaError_t launch_pack_level(const float *src, void *dst, int Nx, int Ny, int Nz, int pz,
                              int storage, float inv_scale, cudaStream_t s);
// u^{n-1} = u^n - d^n of a 16-bit shot into dense FP32
cudaError_t launch_unpack_prev(const void *u, const void *d, float *dst, int Nx, int Ny, int Nz, int pz,
                               int storage, const LevelScales *scales, int slot, cudaStream_t s);
cudaError_t launch_set_level_scale(LevelScales *scales, int slot, float scale, unsigned amax_bits,
                                   float dscale, unsigned damax_bits, cudaStream_t s);

}  // namespace fdgb
