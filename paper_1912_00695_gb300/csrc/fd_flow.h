// Flow schedule of the single-step TMA kernel (see fd_flow.cuh): the
// arguments of one persistent launch that advances nt time steps.
#pragma once
#include <cuda_runtime.h>

#include "fd_internal.h"

namespace fdgb {

struct FlowArgs {
    TmaMaps maps[2];    // maps of a step whose u^n is buffer 0 / buffer 1
    StepArgs a[2];      // step arguments with u^n in buffer 0 / buffer 1 (step field unused)
    long long step0;    // global index of the first step
    int nt;             // steps of this launch
    int cur0;           // buffer holding u^{step0}
    int nbz, nby, nbx;  // tiles along z, y and x-chunks: work items per step = nbz nby nbx
    // zeroed before the launch: the work counter, the abort word, then one flag
    // per (tile, x-chunk) = the number of this launch's steps it has completed
    int *counter;
    unsigned *abort;
    unsigned *flags;
    // BF16 storage: the launch stores every level it writes with unit scales (BF16
    // has FP32's exponent range, so a power-of-two scale changes no rounding);
    // the first step reads the levels' own scales from the handle's slots, and
    // the maxima of every stored value land in amax[0] (u) and amax[1] (d), zeroed
    // with the flags, for the next launch's scale selection
    unsigned *amax;
    // FP32 only, null / zero otherwise. Regions are numbered as the flags.
    // Receivers: the item of step s samples its input level u^{step0+s} at the
    // receivers of its region (entries rec_start[rem] .. rec_start[rem + 1] - 1:
    // trace row rec_row, the pitched offset rec_off of the lower corner node and
    // 8 weights rec_w in the corner order of the receivers' own tables) into
    // traces[row * rec_stride + (step0 + s - rec_s0 - 1)] when that index lies in
    // [0, rec_stride). Sources beyond the fused ones: the item of step s adds the
    // sources of its region (entries xs_start[rem] ..: source index xs_idx and
    // pitched node offset xs_off, in source order) to u^{step0+s+1} after its
    // own stores, one thread per entry when the nodes are pairwise distinct
    // (xs_distinct), else one thread in order.
    const int *rec_start, *rec_row;
    const long long *rec_off;
    const float *rec_w;
    float *traces;
    int rec_stride;
    long long rec_s0;
    const int *xs_start, *xs_idx;
    const long long *xs_off;
    int xs_distinct;
};

// Flow schedule of a batch (FP32): one persistent launch advances every shot of
// the batch by nt steps. Work items (step s, work-list entry w) are numbered
// step-major; an item waits for the 27 items of step s - 1 around it in its
// own shot (x-chunks, y and z tiles +-1), as the single-shot flow does.
struct BatchFlowArgs {
    const BatchShot *shots;  // per shot: arguments and maps for both buffer parities, cur0, step0
    const int4 *items;       // work list: (shot, bz, by, bx); each shot's entries contiguous,
                             // x-chunk slowest and z tile fastest
    const int4 *geo;         // per shot: (z tiles, y tiles, x-chunks, index of its first entry)
    int n_items;             // work-list entries (items per step)
    int nt;                  // steps of this launch
    // zeroed before the launch: the work counter, the abort word, then one flag per
    // work-list entry = the number of this launch's steps it has completed
    int *counter;
    unsigned *abort;
    unsigned *flags;
};

// One persistent batch launch (radius <= 8, FP32, batch tiles); cudaErrorInvalidValue
// for a configuration without one.
cudaError_t launch_tma_batch_flow(int radius, int form, int tile_z, int tile_y, const BatchFlowArgs &f, int ctas,
                                  cudaStream_t s);
// Resident CTAs per SM of that kernel (0 if the configuration does not exist).
int tma_batch_flow_ctas_per_sm(int radius, int form, int tile_z, int tile_y);

// One persistent launch of the flow kernel for radius/form/tile; `ctas` is the
// number of CTAs (at most the resident count). cudaErrorInvalidValue for a
// configuration without a flow kernel.
cudaError_t launch_tma_flow(int radius, int form, int storage, int tile_z, int tile_y, int rows, const FlowArgs &f,
                            int ctas, bool check, cudaStream_t s);
// After a BF16 flow launch: the level it ended on gets unit scales and the
// launch's maxima (the next per-step launch selects its scales from them).
cudaError_t launch_flow_finish_scales(LevelScales *scales, int slot, const unsigned *amax, cudaStream_t s);
// Resident CTAs per SM of that kernel (0 if the configuration does not exist);
// ex: the FP32 variant with receivers and extra sources (launched when the
// arguments carry their tables).
int tma_flow_ctas_per_sm(int radius, int form, int storage, int tile_z, int tile_y, int rows, bool ex);

}  // namespace fdgb
