/*
 * fd_acoustic.h — C-ABI of a GB300 (sm_103a) library for the explicit time step
 * of the 3D acoustic isotropic wave equation with absorbing-layer damping and
 * point-source injection (arXiv 1912.00695):
 *
 *   m u_tt - Lap u + eta u_t = q,   u(.,0) = 0,  u_t(.,0) = 0          (Sec. 2.1, Eq. 1)
 *
 * with m = 1/c^2 the squared slowness, eta >= 0 the damping of the absorbing
 * layer (the `damp` field of Listing 2) and q the point sources. Time is
 * discretised by the second-order leapfrog (Listing 1: time_order=2) and the
 * Laplacian by the central finite-difference stencil of accuracy order k
 * (Listing 1: space_order = k, stencil radius r = k/2), so one step is
 *
 *   u^{n+1} = (dt^2 (L u^n + q^n) + m (2u^n - u^{n-1}) + dt/2 eta u^{n-1}) / (m + dt/2 eta),
 *
 * the form Listing 2 prints for k = 2 (there with h = 1 and every term divided
 * by r0 = dt m + dt^2/2 damp).
 *
 * Conventions shared by every call:
 *  - Grid. nx, ny, nz count the interior; the computational domain adds nbl
 *    absorbing cells on each side: N_a = n_a + 2 nbl. Host and device arrays
 *    are dense C-order [x][y][z] over the computational domain (z fastest),
 *    the order Listing 2 indexes u[t][x][y][z]. Beyond the computational
 *    domain the field is zero (Dirichlet).
 *  - Errors. Every call returns FD_OK (0) or a negative FD_E* code; the text
 *    of the last error of the calling thread is available from
 *    fd_last_error(). No C++ exception crosses the ABI.
 *  - Ownership. Host arrays passed in are copied; the caller keeps them. The
 *    library owns the device buffers of a handle until fd_destroy().
 *  - Threading and streams. A handle is not thread-safe. Its work is queued
 *    on one CUDA stream (fd_set_stream; default: a blocking stream the handle
 *    creates, which orders with the legacy default stream).
 *    Calls that return data to the host synchronise that stream.
 */
#ifndef FD_ACOUSTIC_H
#define FD_ACOUSTIC_H

#ifdef __cplusplus
extern "C" {
#endif

/* ---- status codes -------------------------------------------------------- */
#define FD_OK 0
#define FD_EINVAL (-1)      /* an argument is out of its documented range         */
#define FD_ERANGE (-2)      /* a source node lies outside the interior            */
#define FD_EUNSTABLE (-3)   /* dt exceeds the stability limit of the model        */
#define FD_ENOMEM (-4)      /* a device or host allocation failed                 */
#define FD_ECUDA (-5)       /* a CUDA runtime call failed                         */
#define FD_ENONFINITE (-6)  /* the wavefield reached NaN/Inf (or 16-bit overflow) */
#define FD_ETIMEOUT (-7)    /* a bounded device-side wait ran out (reported by
                               fd_synchronize / fd_read_wavefield)                */
#define FD_ESTATE (-8)      /* call out of order, e.g. fd_forward before a model  */
#define FD_ENOTSUP (-9)     /* option combination not supported                   */
#define FD_EFULL (-10)      /* batch/server: no slot or memory budget left        */

/* ---- options -------------------------------------------------------------- */
/* Storage precision of the wavefields (the Laplacian and the update are
 * always computed in FP32; m and eta stay FP32). FP32 keeps the two leapfrog
 * levels u^n, u^{n-1}. The 16-bit formats keep u^n and the increment
 * d^n = u^n - u^{n-1}, each with its own per-level power-of-two scale, and
 * step d^{n+1} = dt^2/(m + dt/2 eta) (L u^n + q) + (1 - dt eta/(m + dt/2 eta)) d^n,
 * u^{n+1} = u^n + d^{n+1} (the same scheme, rearranged): rounding both levels
 * instead would lose the small difference u^n - u^{n-1} and drift without
 * bound over long runs. 16-bit storage needs the factored form. */
#define FD_STORAGE_F32 0
#define FD_STORAGE_BF16 1   /* bfloat16 u and increment, per-level power-of-two scales */
#define FD_STORAGE_F16 2    /* float16 u and increment, per-level power-of-two scales  */

/* Symbolic form of the stencil expression (Sec. 4: Devito's "basic" versus
 * "aggressive" symbolic optimisation). Both compute the same update. */
#define FD_FORM_FACTORED 0  /* common factors hoisted, equal-distance taps summed first,
                               dt^2/(m + dt/2 eta) precomputed per point */
#define FD_FORM_EXPANDED 1  /* every tap multiplied by its own coefficient and divided
                               by (m + dt/2 eta) per point, as Listing 2 is written (the
                               division as a multiply by the hardware's approximate
                               reciprocal, within 1 ulp, taken once per point and step) */

/* Kernel schedule. */
#define FD_KERNEL_AUTO 0    /* the TMA kernel, launch shape chosen by the autotuner */
#define FD_KERNEL_STREAM 1  /* 2.5D streaming kernel, one point per thread (x-march, y-z tile
                               staged through registers into shared memory); FP32 only */
#define FD_KERNEL_NAIVE 2   /* one thread per point, all taps from global memory; FP32 only */
#define FD_KERNEL_TMA 3     /* 2.5D streaming kernel, four z points per thread, y-z tile with
                               halo fetched by tensor-map bulk copies; FP32 storage (both
                               forms) and 16-bit storage (factored form) */

/* Outer boundary of the computational domain (the paper gives none; Sec. 2
 * names absorbing layers only). */
#define FD_BOUNDARY_ZERO 0      /* zero (Dirichlet) halo of k/2 cells: the solver's mode  */
#define FD_BOUNDARY_PERIODIC 1  /* every axis wraps around (a 3-torus): a test mode in
                                   which the scheme's discrete plane waves and, with
                                   eta = 0, its discrete energy are known exactly; FP32,
                                   naive kernel, single shots only                        */

typedef struct fd_options {
    int storage;       /* FD_STORAGE_*                                             */
    int form;          /* FD_FORM_*                                                */
    int kernel;        /* FD_KERNEL_*                                              */
    int tile_z;        /* tile width along z: STREAM 32; TMA 32, 64 or 128; 0 = autotune */
    int tile_y;        /* tile rows along y: STREAM 4, 8, 16; TMA (FP32) with tile_z 32:
                          16 or 32, 64: 8 or 16, 128: 8; TMA (16-bit) 32x16 or 64x8;
                          space orders 18-24 (TMA): 32x16 or 32x32 (FP32), 32x16
                          (16-bit); 0 = autotune                                    */
    int x_block;       /* planes per CTA along x (each CTA streams x_block
                          consecutive planes of one y-z tile); 0 = autotune         */
    int check_finite;  /* 1 = fold a max|u| reduction into each step so that
                          fd_read_wavefield/fd_status report FD_ENONFINITE          */
    int boundary;      /* FD_BOUNDARY_*                                            */
    int rows;          /* TMA kernel: y rows per thread, 1 or 2 (space orders <= 16;
                          two rows share the y-tap loads: tiles 32x32 and 64x16,
                          tile_y counting every row); 0 = autotune                  */
} fd_options;

typedef struct fd_handle fd_handle;

/* Fill *opt with the defaults: FP32, factored, auto kernel, autotuned tile
 * and x_block, finite check on, zero boundary. */
void fd_options_default(fd_options *opt);

/* ---- single-shot solver --------------------------------------------------- */

/* Create a solver for an nx*ny*nz interior with an nbl-cell absorbing layer on
 * every side, space order k (even, 2..24), grid spacing h and time step dt
 * (both > 0, any consistent units). Allocates the device state (two wavefield
 * levels, the model fields) and zeroes the wavefields (Eq. 1: u = u_t = 0 at
 * t = 0). FD_EINVAL when k is odd or outside [2,24], n_a < 1, nbl < 0, a
 * computational extent N_a exceeds 65535, or h, dt are not positive finite;
 * FD_ENOMEM when the device buffers do not fit. *out is NULL on failure.
 * Any N_a >= 1 is a valid shot: taps beyond the domain read the zero halo,
 * so a domain thinner than the stencil (down to one node) needs no special
 * case. */
int fd_acoustic_create(int nx, int ny, int nz, int space_order, double h, double dt, int nbl,
                       fd_handle **out);

/* As fd_acoustic_create with explicit options (opt == NULL: defaults).
 * FD_ENOTSUP for an unknown storage/form/kernel/boundary value, 16-bit
 * storage with the expanded form or a kernel other than TMA/AUTO, a
 * (tile_z, tile_y) pair the chosen kernel does not have, or the periodic
 * boundary with 16-bit storage or a kernel other than NAIVE/AUTO (AUTO then
 * selects NAIVE). */
int fd_acoustic_create_ex(int nx, int ny, int nz, int space_order, double h, double dt, int nbl,
                          const fd_options *opt, fd_handle **out);

/* Set the model from HOST arrays over the computational domain
 * (N_x*N_y*N_z floats, C-order): m = 1/v^2 (> 0, finite) and eta (>= 0,
 * finite). eta == NULL selects the default absorbing profile
 *   eta = m * sum_a d_max (l_a / nbl)^2,  d_max = 3 v_max ln(1000) / (2 nbl h),
 * l_a the depth (in cells) into the layer along axis a, v_max = 1/sqrt(min m)
 * (a convention: the paper names absorbing boundaries but gives no profile).
 * Checks stability: FD_EUNSTABLE when dt > fd_dt_max(k, h, v_max).
 * FD_EINVAL for non-positive or non-finite m, negative or non-finite eta.
 * Validation, the default profile and the derived per-point coefficients run
 * on the device after one copy of m (and eta); on failure the handle has no
 * model (fd_forward returns FD_ESTATE) until a valid one is set. Resets
 * nothing: the wavefields keep their state. */
int fd_set_model(fd_handle *hd, const float *m, const float *eta);

/* As fd_set_model, from DEVICE arrays of the same layout (e.g. a torch
 * tensor's data_ptr()), copied device-to-device on the handle's stream. */
int fd_set_model_device(fd_handle *hd, const float *d_m, const float *d_eta);

/* Add a point source at INTERIOR node (ix, iy, iz) (offset by nbl internally)
 * with nt samples: q^n = wavelet[n] for global steps n < nt, 0 afterwards
 * (the q_s of Eq. 1, entering the update as dt^2 q / (m + dt/2 eta) at that
 * node). Several sources add up. The wavelet is copied. FD_ERANGE when the node
 * is outside the interior; FD_EINVAL when nt < 1 or wavelet is NULL. */
int fd_inject(fd_handle *hd, int ix, int iy, int iz, const float *wavelet, int nt);

/* Remove every source. */
int fd_clear_sources(fd_handle *hd);

/* Sources and receivers between nodes: the next step of the workflow after
 * the forward step (Sec. 5 names receivers and the imaging workflow as future
 * work; no formula is given). Coordinates are continuous INTERIOR coordinates
 * in grid units: interior node (i, j, l) sits at (i, j, l), and each
 * coordinate must lie in [0, n_a - 1] of its axis (FD_ERANGE otherwise; NaN
 * included). A point belongs to the cell with lower node
 * i0 = min(floor(t), N - 2) on each axis (domain index t = coordinate + nbl),
 * and its 8 corner weights are the trilinear W_c = prod_a (1 - |t_a - c_a|).
 *
 * fd_inject_at: an off-grid point source, spread onto the nodes of its cell:
 * each corner with W_c > 0 becomes one point source (as fd_inject) whose
 * wavelet is W_c times the given one, rounded to FP32 (so up to 8 sources per
 * call). Spreading is the transpose of the receivers' sampling, which keeps
 * source-receiver reciprocity. Same errors as fd_inject. */
int fd_inject_at(fd_handle *hd, double x, double y, double z, const float *wavelet, int nt);

/* Receivers: n points at xyz[3r], xyz[3r+1], xyz[3r+2] (host array, copied),
 * replacing any earlier set (n = 0 removes them). From the handle's current
 * step s0 on, every step records per receiver the trilinear interpolation
 * sum_c W_c u^{n+1}[c] of the level it has just written (after source
 * injection; 16-bit storage: dequantised with that level's scale): sample i of
 * receiver r is u^{s0+i+1} there, stored at traces[r * nt_max + i], for
 * i < nt_max; later steps are not recorded. fd_reset restarts the traces at
 * step 0, fd_load_state at the loaded step. Device memory: 8 (offset, weight)
 * pairs per receiver and n * nt_max floats, owned by the handle. FD_EINVAL for
 * n < 0, a NULL xyz or nt_max < 1 with n > 0, or n * nt_max > 2^31; FD_ERANGE
 * for a point outside the interior; FD_ENOMEM. */
int fd_set_receivers(fd_handle *hd, int n, const double *xyz, int nt_max);

/* FWI gradient of one shot (the adjoint workflow the paper names as its
 * motivation, Sec. 1 and Sec. 5; FP32 storage, factored form, TMA kernel).
 * Runs the handle's shot (its sources, from step 0: the handle is reset and
 * ends at step nt with these receivers set) for nt steps, records the traces
 * d^n = R u^{n+1} at the nrec receivers (rec_xyz as fd_set_receivers), and
 * returns the misfit J = 1/2 sum (d - d_obs)^2 (FP64 sum) and its exact
 * discrete gradient with respect to m (eta held fixed):
 *   dJ/dm = - sum_{n<nt} w^{n+1} (u^{n+1} - 2u^n + u^{n-1}),
 * w the adjoint field: the same step run backward in time from
 * w^{nt+1} = w^{nt+2} = 0 with the residuals injected at the receivers
 * (spreading = transpose of the sampling). The forward pass stores the second
 * time difference of every step in device memory (nt fields of the pitched
 * size: FD_ENOMEM if it does not fit), fused into the step kernel; the adjoint
 * pass accumulates the gradient in its step kernel. d_obs: HOST [nrec][nt];
 * grad_out: HOST N_x*N_y*N_z floats (C-order, whole domain); syn_out: HOST
 * [nrec][nt] synthetic traces or NULL. FD_EINVAL/FD_ERANGE for bad
 * arguments, FD_ESTATE without a model, FD_ENOTSUP for other storage/form/
 * kernel choices. Synchronises; fd_last_forward_ms then returns the device
 * time of the two passes (which run back to back: the residual is formed on
 * the device). When the history does not fit in 80 % of the free device
 * memory, the call checkpoints instead (as fd_fwi_gradient_checkpointed with
 * segment = ceil(sqrt(nt))). */
int fd_fwi_gradient(fd_handle *hd, int nrec, const double *rec_xyz, const float *d_obs, int nt, float *grad_out,
                    float *syn_out, double *misfit);

/* As fd_fwi_gradient with wavefield checkpointing: the forward pass keeps only
 * the states (u^j, u^{j-1}) at j = 0, segment, 2 segment, ...; the adjoint
 * pass recomputes each segment's history from its checkpoint just before it
 * is needed (one extra forward pass; device memory about 2 nt/segment +
 * segment + 4 fields instead of nt + 4). The recomputation repeats the same
 * per-point arithmetic, so the gradient, traces and misfit equal those of
 * fd_fwi_gradient bit for bit. segment >= nt is the full history; FD_EINVAL
 * for segment < 1. */
int fd_fwi_gradient_checkpointed(fd_handle *hd, int nrec, const double *rec_xyz, const float *d_obs, int nt,
                                 int segment, float *grad_out, float *syn_out, double *misfit);

/* As fd_forward, two time steps per launch (temporal blocking along the
 * streaming direction: the next step of the paper's data-locality argument,
 * Sec. 5): each launch reads u^n, u^{n-1}, w (and eta's coefficient in the
 * layer) once and writes u^{n+1} and u^{n+2}, computing the intermediate level
 * on overlapping extended tiles; an odd last step runs the single-step
 * kernel. Same results bit for bit as fd_forward (same per-point arithmetic).
 * FP32 storage, factored form, space order 2 or 4, at most 4 sources, no
 * receivers (FD_ENOTSUP otherwise). Allocates two more wavefield buffers on
 * first use; the handle's state then rotates through the four buffers.
 * Asynchronous like fd_forward. fd_forward itself takes this path for space
 * order 2 when the kernel is left to the library (FD_KERNEL_AUTO) and the
 * conditions hold. */
int fd_forward_two_step(fd_handle *hd, int nt);

/* As fd_forward with one persistent launch for the nt steps instead of one
 * launch per step (the flow schedule): work items (step, y-z tile, x-chunk)
 * are taken in step order by resident CTAs, and an item starts as soon as the
 * 27 items of the previous step around it are done, so the SMs do not idle in
 * the tail of each step and between launches. Same per-point arithmetic as
 * fd_forward with the TMA kernel: the same results bit for bit. FP32 storage
 * (BF16 with at most 4 sources and no receivers), the TMA kernel (either
 * form), zero boundary, x_block >= k/2 (FD_ENOTSUP otherwise). With FP32,
 * receivers and sources beyond the 4 fused ones ride on the items: an item
 * samples its input level at the receivers whose lower trilinear corner lies
 * in its region, and adds the extra sources of its region (in their order)
 * after its stores, so traces and fields equal the per-step launches' bit for
 * bit; the per-region lists are built on the host and kept on the device
 * (rebuilt when the x-chunk, the tile, the sources or the receivers change).
 * A device-side wait that
 * gives up (about 2 s) ends the launch and sets FD_ETIMEOUT in the status.
 * The x-chunk length is the options' x_block if set, else timed on the
 * first steps of the first call of at least 144 steps for the grid and launch
 * shape (candidates 8-64 planes, 8 steps each; all of them part of the
 * requested steps, same bits) and cached for the process; a shorter first
 * call uses 40 planes for that call only. The same first call compares the
 * two schedules by the cost of one more step: the best length and the
 * per-step launches each run 8 and 24 steps, and (t24 - t8) / 16 is compared,
 * which cancels a launch's start-up and last tail.
 * fd_forward takes this path when the kernel is left to the library
 * (FD_KERNEL_AUTO), the conditions hold, the two-step path (space order 2,
 * factored) does not apply and that comparison did not find the per-step
 * launches cheaper per step for the grid.
 * Asynchronous like fd_forward; fd_last_forward_ms times the launch. */
int fd_forward_flow(fd_handle *hd, int nt);

/* Copy the traces into HOST memory out[n * nt_max] (r-major; samples not yet
 * recorded are zero) and the number of recorded samples per receiver into
 * *recorded. Synchronises the handle's stream; returns the device status like
 * fd_synchronize. FD_ESTATE when no receivers are set. */
int fd_read_traces(fd_handle *hd, float *out, int *recorded);

/* Queue nt time steps on the handle's stream (asynchronous; returns before
 * the GPU finishes). Each step is the explicit leapfrog update of Eq. 1 with
 * the damping term of Listing 2 (its r0 = dt m + dt^2/2 damp denominator) and
 * the point sources' q_s, over the three time levels that Listing 2 names
 * t0, t1, t2 (Sec. 2.1); the paper's measured runs repeat it 30,000 times
 * (Sec. 4). The global step counter persists across calls, so
 * fd_forward(a) followed by fd_forward(b) equals fd_forward(a + b) bit for
 * bit. Steps are replayed from a cached CUDA graph. With the kernel left to
 * the library, FP32 shots run the flow schedule (fd_forward_flow) or, at
 * space order 2 factored without receivers, two steps per launch
 * (fd_forward_two_step); every schedule gives the same bits. FD_ESTATE
 * without a model; FD_EINVAL for nt < 0. */
int fd_forward(fd_handle *hd, int nt);

/* Copy a wavefield level to a HOST array of N_x*N_y*N_z floats (dense C-order;
 * Sec. 5 names returning the result to the host workflow as future work, so
 * the paper defines no read-back format; 16-bit storage is converted and scaled to FP32). level 0 = u^n (the newest),
 * 1 = u^{n-1}. Synchronises the stream. Returns FD_ENONFINITE when the finite
 * check saw NaN/Inf (or 16-bit overflow) in any step since the last reset. */
int fd_read_wavefield(fd_handle *hd, float *out, int level);

/* As fd_read_wavefield into a DEVICE array (N_x*N_y*N_z floats); queued on the
 * handle's stream, returns without synchronising (status not checked). */
int fd_read_wavefield_device(fd_handle *hd, float *d_out, int level);

/* (The paper has no counterpart: stream binding is this library's host
 * runtime.) Bind the handle to a CUDA stream (a cudaStream_t, e.g. torch's
 * torch.cuda.current_stream().cuda_stream); NULL = the handle's own stream
 * (created blocking, so it orders with the legacy default stream). Waits for
 * the work already queued on the previous stream. */
int fd_set_stream(fd_handle *hd, void *cuda_stream);

/* Wait for the handle's queued work; returns the device status (FD_OK,
 * FD_ENONFINITE) or FD_ECUDA. (The paper has no counterpart: status and
 * synchronisation are this library's host runtime.) */
int fd_synchronize(fd_handle *hd);

/* Device status without waiting beyond what is queued: same as fd_synchronize. */
int fd_status(fd_handle *hd);

/* Load the solver state from HOST arrays over the computational domain
 * (N_x*N_y*N_z floats each, dense C-order): u = u^step (level 0) and
 * u_prev = u^{step-1} (level 1), and set the global step counter to `step`
 * (>= 0; it indexes the source wavelets). Together with fd_read_wavefield and
 * fd_get_step this is checkpoint/resume. 16-bit storage stores u and
 * u - u_prev with power-of-two scales picked from their max magnitudes. Clears
 * the device status.
 * FD_EINVAL for NULL arrays, non-finite values or step < 0. */
int fd_load_state(fd_handle *hd, const float *u, const float *u_prev, long long step);

/* Zero both wavefield levels, the step counter and the device status: the
 * zero initial conditions u = u_t = 0 of Eq. 1 (Sec. 2.1). Keeps the model
 * and the sources. Queued on the handle's stream (asynchronous). */
int fd_reset(fd_handle *hd);

/* Global step counter n (the wavefield level u^n held as level 0). */
int fd_get_step(fd_handle *hd, long long *step);

/* Computational-domain extents N_x, N_y, N_z of a handle. */
int fd_get_dims(fd_handle *hd, int *Nx, int *Ny, int *Nz);

/* Launch configuration the handle uses for its step kernel (FD_KERNEL_* id,
 * tile_z, tile_y, x_block): what the autotuner picked or the options forced
 * (zeros before the first fd_forward when the autotuner still has to run). */
int fd_get_config(fd_handle *hd, int *kernel, int *tile_z, int *tile_y, int *x_block);

/* The schedule fd_forward runs for this handle: *rows = y rows per thread of
 * the TMA kernel; *schedule = 0 one launch per step, 1 the flow schedule (one
 * persistent launch per call), 2 two steps per launch; *flow_x_block = the
 * flow schedule's x-chunk (0 until chosen). Zeros before the first fd_forward
 * when the autotuner still has to run. Any pointer may be NULL. (The paper has
 * no counterpart: launch shapes are this library's.) */
int fd_get_schedule(fd_handle *hd, int *rows, int *schedule, int *flow_x_block);

/* Device time of the step kernels queued by the last fd_forward (or
 * fd_forward_two_step), in ms, measured by CUDA events on the handle's stream
 * around the graph replay or the two-step launches (synchronises). FD_ESTATE
 * if no fd_forward was timed yet. */
int fd_last_forward_ms(fd_handle *hd, float *ms);

/* Number of this library's kernel launches executed or queued since it was
 * loaded, over all handles, batches and fd_forward_noalloc calls: a replayed
 * CUDA graph adds the kernels it holds (launches recorded into a graph are not
 * counted when recorded). The difference of two readings counts the launches
 * of the span between them. No device work; FD_EINVAL if count is NULL. */
int fd_kernel_launches(long long *count);

/* Release every device buffer and the handle. NULL is accepted (no-op).
 * (The paper has no counterpart: buffer ownership is this library's.) */
int fd_destroy(fd_handle *hd);

/* ---- batches of uneven shots ---------------------------------------------- */
/* A batch advances many independent shots (each its own grid, model, dt and
 * sources; all with the same space order, h, storage and form) together: one
 * kernel launch per time step covers every shot's tiles, or (FP32, when the
 * autotuner finds it cheaper, or on request) one persistent launch covers
 * every step of a forward, and the launches are replayed from a CUDA graph.
 * Shots keep their own step counters, so shots
 * added later run behind the others; a shot's result does not depend on which
 * other shots share the batch (same arithmetic per point as fd_forward). Each
 * shot is the time step of Sec. 2.1, Eq. 1 (see the top of this header). */
typedef struct fd_batch fd_batch;

/* Device bytes one shot of this size needs (wavefields, model fields, small
 * buffers), for admission by memory budget. storage: FD_STORAGE_*. */
int fd_shot_device_bytes(int nx, int ny, int nz, int nbl, int storage, long long *out);

/* Create an empty batch of space order k (even, 2..16: FD_EINVAL otherwise).
 * opt: storage/form as for fd_acoustic_create_ex
 * (16-bit storage needs the factored form), tile_z/tile_y 0 (autotuned) or
 * one of 32x16, 64x8; x_block 0 (autotuned) or the planes per CTA of every
 * shot (the whole extent if shorter); rows 0 or 1; kernel FD_KERNEL_TMA pins
 * one launch per step (no schedule probes), any other value lets FP32
 * batches choose their schedule.
 * FD_ENOTSUP for other shapes. The autotuner (the batch counterpart of the
 * loop blocking and auto-tuning Devito applies, Sec. 5) times the launch
 * shapes not forced — both tiles, x-chunks of 32/48/64/96/128 planes and whole
 * extents — on 3 real steps each of the first fd_batch_forward of at least
 * 39 steps (9 with a forced x_block) over at least 4 shots, and keeps the
 * fastest for the batch's lifetime (shots added later take it); before that,
 * 96-plane chunks. FP32 batches then (on that forward if 30 steps remain,
 * else on the next forward of at least 30 steps; 27 with a forced x_block)
 * time the persistent launch (fd_batch_forward_flow) on the chosen tile at the
 * chosen x-chunks and at 48-plane chunks, and compare the cost of one more
 * step of each schedule ((9-step time - 3-step time) / 6) to pick the schedule
 * fd_batch_forward runs. Results do not depend on the shape or the schedule
 * (same arithmetic per point). */
int fd_batch_create(int space_order, double h, const fd_options *opt, fd_batch **out);

/* Add a shot: interior nx*ny*nz, layer nbl, time step dt, HOST model m and
 * eta (eta NULL: default profile) exactly as fd_acoustic_create +
 * fd_set_model (same errors). Allocates its device state (see
 * fd_shot_device_bytes). *slot receives its id (slots of removed shots are
 * reused). The shot starts at step 0 with zero wavefields. */
int fd_batch_add(fd_batch *b, int nx, int ny, int nz, int nbl, double dt, const float *m,
                 const float *eta, int *slot);

/* Source of a shot, as fd_inject (at most 4 sources per batched shot:
 * FD_ENOTSUP beyond). */
int fd_batch_inject(fd_batch *b, int slot, int ix, int iy, int iz, const float *wavelet, int nt);

/* Remove a shot and free its device memory (waits for queued work). */
int fd_batch_remove(fd_batch *b, int slot);

/* Advance every shot in the batch by nt steps (asynchronous, on the batch's
 * stream), with the schedule the autotuner chose (one launch per step until
 * it has run). Each step is Sec. 2.1, Eq. 1 for every shot. */
int fd_batch_forward(fd_batch *b, int nt);

/* As fd_batch_forward, in one persistent launch (FP32 storage; FD_ENOTSUP
 * otherwise): resident CTAs claim (step, work item) pairs step-major and an
 * item of step s starts once the 27 items of step s - 1 around it in its own
 * shot are done (flags in device memory, waits bounded by the global timer:
 * a wait that runs out sets FD_ETIMEOUT in that shot's status). The paper
 * runs one kernel per step (Sec. 4); this schedule is the batch counterpart
 * of the single-shot flow schedule. Same results bit for bit. */
int fd_batch_forward_flow(fd_batch *b, int nt);

/* *flow = 1 when fd_batch_forward runs the persistent launch (FP32, chosen by
 * the autotuner), 0 for one launch per step. (The paper has no counterpart.) */
int fd_batch_schedule(fd_batch *b, int *flow);

/* Read a shot's wavefield level (as fd_read_wavefield / _device). */
int fd_batch_read(fd_batch *b, int slot, float *out, int level);
int fd_batch_read_device(fd_batch *b, int slot, float *d_out, int level);

/* A shot's global step counter; a shot's device status (as fd_status). */
int fd_batch_shot_step(fd_batch *b, int slot, long long *step);
int fd_batch_shot_status(fd_batch *b, int slot);

/* The batch's launch shape: tile, x-chunk policy (planes per CTA, 0 = whole
 * extents) and whether the autotuner has run or the shape was forced (any
 * pointer may be NULL). (The paper has no counterpart.) */
int fd_batch_get_config(fd_batch *b, int *tile_z, int *tile_y, int *x_block, int *tuned);

/* Number of shots in the batch and work items (CTAs) per step (-1 until the
 * next fd_batch_forward rebuilds the work list). */
int fd_batch_size(fd_batch *b, int *active, int *work_items);

/* Zero every shot's wavefields, step counter and status (as fd_reset). */
int fd_batch_reset(fd_batch *b);

/* Stream binding and synchronisation of the batch (as for handles). */
int fd_batch_set_stream(fd_batch *b, void *cuda_stream);
int fd_batch_synchronize(fd_batch *b);

/* Free every shot and the batch. NULL is accepted. */
int fd_batch_destroy(fd_batch *b);

/* ---- slabs: one shot split along x ---------------------------------------- */
/* The paper's OPS backend partitions a block across a distributed-memory set
 * of processes (Sec. 3, Devito-OPS integration, item (vii): ops_partition),
 * and Devito exchanges halos between such subdomains, overlapping the
 * exchange with computation (Sec. 5). A slab is that subdomain for this step:
 * the planes [x0, x1) (computational-domain indices along x, the slowest axis)
 * of one shot, with r = k/2 ghost planes below x0 (if x0 > 0) and above x1 (if
 * x1 < N_x) that hold the neighbouring slabs' values. A step updates only the
 * slab's own planes; its stencil reads the ghost planes, which the caller
 * fills between steps by copying r planes from each neighbour
 * (fd_slab_exchange, or the pointers of fd_slab_exchange_ptrs with any
 * transport). With the ghosts exchanged every step, every point gets the
 * same arithmetic on the same inputs as in the undivided shot: the slabs'
 * planes equal fd_forward's bit for bit.
 *
 * A slab is an fd_handle: fd_set_model (arrays over the slab's buffer: its
 * planes plus ghosts, C-order [x][y][z], N_x = x1 - x0 + ghosts; eta is
 * REQUIRED, since the default profile depends on the whole model),
 * fd_inject (INTERIOR coordinates of the whole shot; a source outside the
 * slab's own planes is ignored, so every slab may be given every source; at
 * most 4 per slab), fd_read_wavefield (the buffer, ghosts included),
 * fd_get_dims, fd_reset, fd_get_step, fd_load_state, fd_set_stream and
 * fd_destroy work as for a shot. fd_forward and the other forward paths,
 * receivers and off-grid sources return FD_ENOTSUP: a slab advances through
 * fd_slab_step. FP32 storage, the TMA kernel, zero boundary (FD_ENOTSUP
 * otherwise); every slab needs at least k/2 own planes (FD_EINVAL). The
 * buffers live on the device current at creation. */

#define FD_SLAB_BOUNDARY 1 /* the own planes within r of a neighbour (they read ghost planes) */
#define FD_SLAB_INTERIOR 2 /* the other own planes; then the step counter advances          */
#define FD_SLAB_ALL 3      /* both                                                          */

/* Create the slab of planes [x0, x1) of an nx*ny*nz (+ nbl layer) shot; the
 * other arguments as fd_acoustic_create_ex. FD_EINVAL for x0 < 0, x1 <= x0,
 * x1 > N_x or fewer than k/2 planes. */
int fd_slab_create(int nx, int ny, int nz, int space_order, double h, double dt, int nbl, int x0, int x1,
                   const fd_options *opt, fd_handle **out);

/* The slab's own planes [*x0, *x1) in domain indices and its ghost plane
 * counts (0 or k/2 each; any pointer may be NULL). A whole shot reports
 * [0, N_x) and no ghosts. */
int fd_slab_info(fd_handle *hd, int *x0, int *x1, int *ghost_lo, int *ghost_hi);

/* Queue part of one time step on the slab's stream. A step is
 * FD_SLAB_BOUNDARY then FD_SLAB_INTERIOR (or FD_SLAB_ALL). Between two steps
 * the ghost planes of the level the step wrote must be filled; the
 * boundary part writes every plane a neighbour needs, so the exchange can run
 * while the interior part computes (overlap of communication with
 * computation). The boundary part of step n+1 reads the ghosts: order the
 * exchange before it (stream order or events). FD_ESTATE without a model. */
int fd_slab_step(fd_handle *hd, int part);

/* Device pointers for the exchange, in the buffer of `level` (0: u^n, the
 * newest level; 1: the other buffer, which the running step writes: between
 * FD_SLAB_BOUNDARY and FD_SLAB_INTERIOR the new values are at level 1, after
 * the step at level 0): send_lo / send_hi = the first / last r own planes
 * (to the lower / upper neighbour's ghosts), recv_lo / recv_hi = the ghost
 * planes below / above; NULL where the slab has no neighbour. *bytes = r
 * planes (r * N_y * pz * 4; pz the padded row pitch). Any output may be NULL. */
int fd_slab_exchange_ptrs(fd_handle *hd, int level, void **send_lo, void **send_hi, void **recv_lo,
                          void **recv_hi, size_t *bytes);

/* Copy the planes of `from` that its x-neighbour `to` needs into `to`'s ghost
 * planes, both at `level`, queued on `stream` (a cudaStream_t; the slabs may
 * live on different devices: a peer copy). FD_EINVAL when the slabs are not
 * neighbours of one shot. */
int fd_slab_exchange(fd_handle *from, fd_handle *to, int level, void *stream);

/* ---- allocation-free stepping -------------------------------------------- */

/* nt time steps on CALLER-OWNED device buffers, allocating no device memory.
 * (The paper has no counterpart: this entry point exists for callers that
 * cannot allocate device memory themselves, such as plug-ins inside a
 * framework whose caching allocator owns the whole device, where a foreign
 * cudaMalloc would bypass its accounting or fail once the pool holds the
 * memory, and latency-bound serving loops, where cudaMalloc/cudaFree would
 * synchronise the device.)
 *
 * Layout: dense C-order [Nx][Ny][Nz] float arrays over the computational
 * domain (no interior/layer split here). d_u = u^{step0}, d_u_prev =
 * u^{step0-1}; each step writes the new level over the older one, so after the
 * call the newest level u^{step0+nt} is in d_u when nt is even and in
 * d_u_prev when nt is odd (the other buffer holds the level before it).
 * d_m = 1/v^2 (> 0), d_eta = damping (>= 0) or NULL for none; both are read
 * as given (no validation, no stability check: the caller owns that). The
 * stencil is the expanded form of fd_forward (same arithmetic per point),
 * space orders 2..16.
 * Sources: ns in [0, 4] point sources at DOMAIN nodes src_xyz (host array,
 * x0,y0,z0, x1,y1,z1, ...), wavelets in the device array d_wavelet (ns rows
 * of ld samples; q = 0 beyond ld), step n uses sample n (global step, from
 * step0). stream: a cudaStream_t (NULL = legacy default stream).
 *
 * Scratch: per-CTA maxima of |u| and the running maximum sit in one static
 * device array of 65,792 bytes (16,384 CTA slots + header) that every GPU
 * loading the library holds until exit. FD_EINVAL when one step would need
 * more than 16,384 CTAs (Ny*Nz above about 4.2 million points) or for bad
 * arguments; FD_ERANGE for a source outside the domain. The first call on a
 * device looks up that device's copy of the array (cudaGetSymbolAddress) and
 * its multiprocessor count (which sizes the x-chunks: four CTAs per
 * multiprocessor) once; make that first call before any stream capture. Every call on a device
 * shares the same array and clears the running maximum at its start, so calls
 * that overlap on the GPU (other streams, other threads) race on it.
 *
 * amax_out (host, may be NULL): when given, the call synchronises the stream,
 * stores max |u| over every point written by the call's steps and returns
 * FD_ENONFINITE if it is NaN/Inf; when NULL the call returns after queueing. */
int fd_forward_noalloc(float *d_u, float *d_u_prev, const float *d_m, const float *d_eta, int Nx,
                       int Ny, int Nz, int space_order, double h, double dt, int ns,
                       const int *src_xyz, const float *d_wavelet, int ld, long long step0, int nt,
                       void *stream, float *amax_out);

/* ---- host numerics -------------------------------------------------------- */

/* Stability limit dt_max = 2 h / (v_max sqrt(3 sum_{j=-r..r} |c_j|)) of the
 * 3D leapfrog scheme (von Neumann analysis at the Nyquist mode). The paper
 * states no limit; this is the classic analysis of the scheme it discretises
 * (Eq. 1, Listing 2), applied to every space order. FD_EINVAL for an odd or
 * out-of-range space order, non-positive h or vmax, or a NULL out. */
int fd_dt_max(int space_order, double h, double vmax, double *out);

/* Centred second-derivative weights c_0..c_r of accuracy order k for unit
 * spacing (out holds k/2 + 1 doubles), computed by Fornberg's recursion.
 * Listing 2 shows k = 2: c_0 = -2, c_1 = 1. */
int fd_fd_weights(int space_order, double *out);

/* The default absorbing-layer damping that fd_set_model uses when eta is NULL,
 * written into the host array eta (Nx*Ny*Nz floats, C-order) for the host
 * model m of the same layout; v_max = 1/sqrt(min m). Host-only helper. */
int fd_default_damping(int Nx, int Ny, int Nz, int nbl, double h, const float *m, float *eta);

/* Text of the calling thread's last error ("" if none). */
const char *fd_last_error(void);

/* Library version string. */
/* Self-test of failure detection on the device (no fault involved): one
 * 32-thread block waits, with the step kernels' own bounded wait functions,
 * on a ring mbarrier whose phase never completes and then on a dependency
 * flag that nothing sets; each wait gives up after its time limit (1 s and
 * 2 s) and the kernel returns, so the context stays usable. *status: bit 0
 * set if the mbarrier wait gave up, bit 1 if the flag wait gave up (3 when
 * both limits work); the seconds each wait lasted go to *mbar_seconds and
 * *flag_seconds (either may be NULL). Synchronises the device (about 3 s).
 * FD_EINVAL if status is NULL, FD_ENOMEM/FD_ECUDA on allocation or launch
 * failure. */
int fd_selftest_waits(unsigned *status, double *mbar_seconds, double *flag_seconds);

const char *fd_version(void);

#ifdef __cplusplus
}
#endif
#endif /* FD_ACOUSTIC_H */
