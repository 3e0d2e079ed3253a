/*
 * wmc.h -- C ABI of the GB300 (sm_103a) Weighted Mean Curvature library.
 *
 * The operations follow Gong & Goksel, "Weighted Mean Curvature", arXiv 1903.07189:
 *   - H^w(U): the "Half Laplace Operator" of Sec. IV-B -- eight signed distances
 *     d_i = h_i * U with the 3x3 half-window kernels h_1..h_8 (Eq. conv), and the one with
 *     the smallest magnitude, H^w = d_m, m = argmin_i |d_i| (Eq. act);
 *   - the explicit, Jacobi-ordered WMC flows that apply it to a whole image:
 *     L2 denoising U^{t+1} = U^t + step (lambda H^w(U^t) - (U^t - f)) (the gradient flow of
 *     Sec. V-B with A = I, where -dR_area/dU is replaced by H^w), and the mean-curvature flow
 *     U^{t+1} = U^t + step H^w(U^t) (Eq. MCF);
 *   - the energies of Eq. wmcr (q = 1) and Eq. 1 (L2 data term), reduced in FP64;
 *   - around them: batches of uneven images, the L1-fidelity primal-dual iteration of Sec. V-C,
 *     the finite-difference discretisation of Eq. rhs that Sec. V-D compares against, and the
 *     reverse mode of unrolled denoising steps and of the energy.
 *
 * Conventions shared by every entry point
 *   Images are single-channel, row-major, h rows by w columns, with a leading dimension
 *   (row pitch) `ld` counted in ELEMENTS (ld >= w).  Element type: see wmc_dtype_t.  Colour
 *   images are processed one channel at a time (the paper does so, Sec. V-D).
 *   Pointers documented as "device" must be CUDA device (or managed) memory readable by the
 *   current device; "host" pointers are ordinary host memory (pinned memory gives
 *   asynchronous copies).  The caller owns every buffer; the library never allocates or
 *   frees memory.  Between calls it keeps only the per-thread error string and, per device,
 *   the kernel attributes it has set (once) and the fixed device array of
 *   wmc_denoise_noalloc.
 *   Work is enqueued on `stream` (NULL = the legacy default stream) and runs asynchronously;
 *   argument errors are detected on the host and returned before anything is enqueued.
 *   No function throws; every failure is a status code, with a detail string available from
 *   wmc_last_error() on the calling thread.
 *   Boundary: WMC_BOUNDARY_REPLICATE reads the nearest in-image pixel outside the image
 *   (a discrete Neumann condition, Sec. III-C / IV-A); WMC_BOUNDARY_ZERO reads 0 there (the
 *   zero padding of the Appendix listing's conv2 'same').
 *   Ties (several d_i of equal magnitude, e.g. on straight ramps) may resolve to either
 *   candidate; every returned value is one of the eight d_i up to FP32 rounding.
 *   Arithmetic is FP32 for every storage type; BF16/FP16 inputs are widened on load and every
 *   stored result (H^w, or U after each step) is rounded to nearest-even.
 */
#ifndef WMC_H
#define WMC_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* Same type as cudaStream_t, declared here so this header needs no CUDA include. */
struct CUstream_st;
typedef struct CUstream_st *wmc_stream_t;

typedef enum {
    WMC_OK = 0,
    WMC_ERR_INVALID_ARG = 1, /* a size, pitch, pointer, dtype, boundary or scalar is invalid */
    WMC_ERR_ALIAS = 2,       /* an output overlaps an input it must not overlap */
    WMC_ERR_UNSUPPORTED = 3, /* valid request this build cannot serve (e.g. no sm_103a GPU) */
    WMC_ERR_CUDA = 4,        /* a CUDA runtime call failed; see wmc_last_error() */
    WMC_ERR_TIMEOUT = 5,     /* a bounded device-side wait gave up (see wmc_denoise_status) */
    WMC_ERR_WORKSPACE = 6    /* workspace missing, too small or misaligned */
} wmc_status_t;

typedef enum { WMC_BOUNDARY_REPLICATE = 0, WMC_BOUNDARY_ZERO = 1 } wmc_boundary_t;

typedef enum { WMC_F32 = 0, WMC_BF16 = 1, WMC_F16 = 2 } wmc_dtype_t;

/* Workspace buffers must start on this many bytes. */
#define WMC_WORKSPACE_ALIGN 256

/*
 * Kernel configuration for the flows.  steps_per_launch = T (1..8) Jacobi steps are taken in
 * on-chip memory per pass over the image (temporal blocking; legal because step t+1 of every
 * pixel reads only U^t, Eq. MCF / Sec. V-B); 0 = library default (4).  tile = the region one CTA
 * updates per step: 1 = 128 x 64 cells (output tiles of 130 - 2T by 66 - 2T), 2 = 128 x 32
 * (130 - 2T by 34 - 2T: less wasted work on small or short images); 0 = library default (1).
 * Results do not depend on the configuration: every configuration performs the same FP32
 * operations on every pixel, so outputs are bitwise identical.
 */
typedef struct {
    int32_t steps_per_launch;
    int32_t tile;
} wmc_config_t;

/* ------------------------------------------------------------------------------------------
 * wmc_eval: H^w(U) at every pixel (Sec. IV-B, Eq. conv + Eq. act).
 *   u   device, h x w, pitch ld_u, type dtype           (input U)
 *   hw  device, h x w, pitch ld_hw, type dtype          (output H^w; must not overlap u)
 *   h, w >= 0 (either 0: nothing to do), ld_u >= w, ld_hw >= w.
 * Errors: WMC_ERR_INVALID_ARG (sizes, null pointer with h*w > 0, bad enum),
 *         WMC_ERR_ALIAS (hw overlaps u), WMC_ERR_CUDA (launch failure).
 */
wmc_status_t wmc_eval(const void *u, void *hw, int32_t h, int32_t w, int64_t ld_u, int64_t ld_hw,
                      wmc_dtype_t dtype, wmc_boundary_t bnd, wmc_stream_t stream);

/* wmc_eval_status: synchronises `stream` and reads, then clears, the library's evaluation status
 * word.  FP32 images that TMA can read (16-byte aligned base and pitch) are evaluated by a
 * persistent kernel that waits for its TMA window loads with a time limit of 0.2 s; a wait that
 * runs out makes that CTA stop (its remaining output is missing) and sets the word, and this
 * returns WMC_ERR_TIMEOUT.  WMC_OK otherwise.  The word is per device and shared by all calls. */
wmc_status_t wmc_eval_status(wmc_stream_t stream);

/* ------------------------------------------------------------------------------------------
 * wmc_denoise: `iters` explicit Jacobi steps of the WMC flow
 *      U^{t+1} = U^t + step * (lambda * H^w(U^t) - mu * (U^t - f)),
 *   mu = 1 when f != NULL (L2 denoising, Sec. V-B with A = I),
 *   mu = 0 when f == NULL (mean-curvature flow, Eq. MCF; lambda then scales the step).
 *   f    device, h x w, pitch ld (observed image) or NULL
 *   u0   device, h x w, pitch ld (U^0) or NULL for U^0 = f; may equal u (resume in place)
 *   u    device, h x w, pitch ld (output U^iters); must not overlap f; if u0 != u it must not
 *        overlap u0 either
 *   lambda finite, >= 0 (regularisation weight, Eq. 1); step finite, > 0 (time step delta,
 *   Eq. MCF -- the paper does not fix it; step*(mu+lambda) <= 1 keeps every iterate inside
 *   the range of f and U^0, a larger step is accepted but carries no such guarantee);
 *   iters >= 0 (0 copies U^0 to u).
 *   workspace: device, >= wmc_denoise_workspace_size() bytes, WMC_WORKSPACE_ALIGN-aligned,
 *   must not overlap f, u0 or u (not needed when iters == 0).  It holds a status word (first
 *   bytes, cleared by every call), one ping-pong image and one flag word per tile of the
 *   multi-step launches (at the end; a call whose chained launches each span more than one
 *   and at most ten waves of CTAs, a wave being two CTAs per SM, clears them first and has a
 *   tile wait for the flags of the tiles of the previous launch that it reads, not for that
 *   whole launch; other calls leave them alone); see wmc_denoise_status().  When the
 *   row pitch is not a multiple of 16 bytes (ld not a multiple of 4 elements for FP32, of 8 for
 *   BF16/FP16) the multi-step kernels cannot read the images through TMA: the workspace then
 *   holds three images of the next aligned pitch, the call copies U^0 and f into two of them,
 *   the launches ping-pong in the workspace and only the last one writes u.
 *   Sides up to 2^24 pixels.
 *   Small images (h <= 256, w <= 256) with iters >= 2 under the default configuration run all
 *   their iterations in ONE launch of one thread-block cluster of ceil(h / 16) CTAs that keep the
 *   image in shared memory (see wmc_denoise_cluster_size); only the status word of the workspace
 *   is then used.  The result is the same bits as the multi-launch path's.
 * Errors: WMC_ERR_INVALID_ARG, WMC_ERR_ALIAS, WMC_ERR_WORKSPACE, WMC_ERR_CUDA.
 */
size_t wmc_denoise_workspace_size(int32_t h, int32_t w, int64_t ld, wmc_dtype_t dtype);

wmc_status_t wmc_denoise(const void *f, const void *u0, void *u, int32_t h, int32_t w, int64_t ld,
                         wmc_dtype_t dtype, float lambda, float step, int32_t iters,
                         wmc_boundary_t bnd, void *workspace, size_t workspace_bytes,
                         wmc_stream_t stream);

/* wmc_denoise_cluster_size: the number of CTAs of the one-launch cluster path that wmc_denoise,
 * wmc_denoise_host and wmc_denoise_noalloc (and wmc_denoise_ex with a NULL or all-zero config)
 * take for an h x w image and `iters` iterations on the current device; 0 when they take the
 * multi-launch path (image larger than 256 x 256, iters < 2, or no such cluster can be scheduled
 * on the device).  Any dtype, either boundary.  Errors: none (negative sizes give 0). */
int32_t wmc_denoise_cluster_size(int32_t h, int32_t w, int32_t iters);

/* As wmc_denoise, with an explicit kernel configuration (NULL = defaults). */
wmc_status_t wmc_denoise_ex(const void *f, const void *u0, void *u, int32_t h, int32_t w,
                            int64_t ld, wmc_dtype_t dtype, float lambda, float step,
                            int32_t iters, wmc_boundary_t bnd, const wmc_config_t *config,
                            void *workspace, size_t workspace_bytes, wmc_stream_t stream);

/* wmc_denoise_status: synchronises `stream` and reads the status word of a workspace last used
 * by wmc_denoise / wmc_denoise_ex / wmc_denoise_host.  The multi-step kernels wait for their
 * asynchronous (TMA) tile loads, and for the flags of the previous launch's tiles they read, with
 * a time limit of 0.2 s; a load wait that runs out makes that CTA skip its tile, a flag wait that
 * runs out lets it go ahead, both set the word, and this returns WMC_ERR_TIMEOUT (the output is
 * then wrong or incomplete).  WMC_OK otherwise.  workspace: device pointer passed to that call. */
wmc_status_t wmc_denoise_status(const void *workspace, wmc_stream_t stream);

/* wmc_selftest_wait_timeout: exercises the failure path of those bounded waits without a fault.
 * One CTA arms an mbarrier for a 16-byte transfer that is never issued and waits for it with the
 * multi-step kernels' bounded wait, limited to limit_ns (1 .. 1e9 ns); the wait runs out and the
 * CTA sets bit 0 of the status word at `workspace`, as a tile whose load timed out does, and
 * returns.  wmc_denoise_status(workspace) then reports WMC_ERR_TIMEOUT; the next flow call on
 * that workspace clears the word.  Nothing but the status word is written.
 *   workspace: device, >= 4 bytes, WMC_WORKSPACE_ALIGN-aligned (a wmc_denoise workspace). */
wmc_status_t wmc_selftest_wait_timeout(void *workspace, int64_t limit_ns, wmc_stream_t stream);

/* wmc_selftest_status_timeout: the same self-test aimed at a status word the library holds per
 * device rather than one in a caller's workspace: target WMC_SELFTEST_EVAL sets the evaluation
 * status word (wmc_eval_status then returns WMC_ERR_TIMEOUT once, and clears it), target
 * WMC_SELFTEST_NOALLOC the word at the start of wmc_denoise_noalloc's fixed scratch array
 * (wmc_denoise_noalloc_status then returns WMC_ERR_TIMEOUT until the next wmc_denoise_noalloc
 * call clears it).  limit_ns as above.  Errors: WMC_ERR_INVALID_ARG (target, limit_ns),
 * WMC_ERR_CUDA. */
/* wmc_selftest_flag_timeout: makes the per-tile flag wait of chained flow launches run out,
 * without a fault.  It runs ONE 4-step flow launch (FP32, lambda 1, step 0.25, replicate
 * boundary, U^0 = f) whose tiles wait for the flags of a previous launch that never ran: the
 * flags are cleared and nothing stores the launch number they wait for.  The first tiles give up
 * after the 0.2 s limit and set the status word; the tiles after them see the word and do not
 * wait.  The launch then computes its 4 steps from f, so u holds the same bits as wmc_denoise with
 * iters = 4, while wmc_denoise_status(workspace) reports WMC_ERR_TIMEOUT until the next flow call
 * on that workspace clears it.
 *   f, u: device, h x w FP32 images of pitch ld; f's start and pitch 16-byte aligned (TMA).
 *   workspace: device, >= wmc_denoise_workspace_size(h, w, ld, WMC_F32) bytes, aligned as above.
 * Errors: WMC_ERR_INVALID_ARG, WMC_ERR_ALIAS, WMC_ERR_WORKSPACE, WMC_ERR_UNSUPPORTED (f not
 * TMA-readable), WMC_ERR_CUDA. */
wmc_status_t wmc_selftest_flag_timeout(const void *f, void *u, int32_t h, int32_t w, int64_t ld,
                                       void *workspace, size_t workspace_bytes, wmc_stream_t stream);

#define WMC_SELFTEST_EVAL 0
#define WMC_SELFTEST_NOALLOC 1
wmc_status_t wmc_selftest_status_timeout(int32_t target, int64_t limit_ns, wmc_stream_t stream);

/* ------------------------------------------------------------------------------------------
 * wmc_denoise_noalloc: wmc_denoise without a workspace argument and without allocating.  It is
 * for callers that cannot obtain device memory for scratch space: code running where a memory
 * pool is owned by someone else and may not be grown, real-time or embedded hosts that forbid
 * allocation after start-up, or bindings that can pass existing image pointers but have no
 * CUDA allocator of their own.  (The paper has no counterpart: this is an interface choice.)
 *   Scratch comes from one fixed device array of wmc_denoise_noalloc_max_bytes() bytes
 *   (32 MiB) inside the library; every GPU that loads the library holds it until the process
 *   exits.  Images whose wmc_denoise_workspace_size() exceeds that are rejected with
 *   WMC_ERR_INVALID_ARG (with a pitch that is a multiple of 16 bytes: FP32 up to about 8.3 M
 *   pixels, e.g. 2880 x 2880; BF16/FP16 up to about 16.7 M, e.g. 4064 x 4064; other pitches
 *   need three images of scratch, so about a third of that) -- use wmc_denoise for larger ones.
 *   The first call on each device looks up the array's device address with that device
 *   current; make that first call before capturing any stream into a CUDA graph.
 *   All calls on a device share the one array and the array keeps the last call's contents:
 *   calls whose work overlaps on the GPU (different streams, or threads enqueueing at the same
 *   time) race and corrupt each other; serialise them (one stream, or events).  The status
 *   word at the start of the array is cleared by every call; a timed-out tile load is reported
 *   by wmc_denoise_noalloc_status() (the counterpart of wmc_denoise_status(), whose workspace
 *   argument such callers do not have).  The array's address is looked up once per device and
 *   kept: do not use the library across a cudaDeviceReset() of that device.  Other arguments,
 *   results and errors: as wmc_denoise.
 */
size_t wmc_denoise_noalloc_max_bytes(void);

/* wmc_denoise_noalloc_status: synchronises `stream` and reads the status word at the start of
 * wmc_denoise_noalloc's fixed scratch array on the current device (as wmc_denoise_status does for
 * a caller's workspace): WMC_ERR_TIMEOUT if a multi-step kernel of the last wmc_denoise_noalloc
 * call on this device gave up waiting for its tile load (its output is then incomplete), WMC_OK
 * otherwise.  The word is cleared by the next wmc_denoise_noalloc call, not by this one. */
wmc_status_t wmc_denoise_noalloc_status(wmc_stream_t stream);

wmc_status_t wmc_denoise_noalloc(const void *f, const void *u0, void *u, int32_t h, int32_t w,
                                 int64_t ld, wmc_dtype_t dtype, float lambda, float step,
                                 int32_t iters, wmc_boundary_t bnd, wmc_stream_t stream);

/* ------------------------------------------------------------------------------------------
 * wmc_denoise_host: wmc_denoise on HOST buffers.  Copies f (and u0) to the device workspace on
 * `stream`, runs the flow there and copies U^iters back into u_host; all of it is enqueued on
 * `stream` and the call returns without waiting (synchronise the stream before reading
 * u_host; pinned host memory makes the copies asynchronous).
 *   f_host  host, h x w, pitch ld (may be NULL for the mean-curvature flow, then u0_host is
 *           required); u0_host host or NULL (U^0 = f); u_host host output, pitch ld.
 *   workspace: DEVICE memory of wmc_denoise_host_workspace_size() bytes (status word first).
 * Errors: as wmc_denoise.
 */
size_t wmc_denoise_host_workspace_size(int32_t h, int32_t w, int64_t ld, wmc_dtype_t dtype);

wmc_status_t wmc_denoise_host(const void *f_host, const void *u0_host, void *u_host, int32_t h,
                              int32_t w, int64_t ld, wmc_dtype_t dtype, float lambda, float step,
                              int32_t iters, wmc_boundary_t bnd, void *workspace,
                              size_t workspace_bytes, wmc_stream_t stream);

/* ------------------------------------------------------------------------------------------
 * wmc_energy: FP64 reductions of one image (Eq. wmcr with q = 1; the L2 data term of Eq. 1):
 *   out[0] = sum_p |H^w(U)(p)|,  out[1] = 1/2 sum_p (U - f)^2,  out[2] = sum_p (U - clean)^2
 *   (out[1] = 0 when f is NULL, out[2] = 0 when clean is NULL).
 *   u, f, clean: device, h x w, pitch ld, type dtype (f, clean may be NULL).  out: DEVICE, 3 doubles, written (not
 *   accumulated).  Sums run in FP32 over at most 16 pixels, then in double-float (an FP32
 *   pair, about 44 bits) up to one warp's share, and in FP64 beyond; the summation order is
 *   fixed by h and w alone, so repeated calls give identical results.  The workspace size
 *   depends on h and w (one FP64 triple per CTA, at most 304 CTAs).  FP32 images that TMA can
 *   read are summed by a kernel fed by TMA copies; if one of its bounded waits (0.2 s) runs out,
 *   out[] holds NaN.
 *   workspace: device, >= wmc_energy_workspace_size() bytes, aligned as above.
 */
size_t wmc_energy_workspace_size(int32_t h, int32_t w);

wmc_status_t wmc_energy(const void *u, const void *f, const void *clean, int32_t h, int32_t w,
                        int64_t ld, wmc_dtype_t dtype, wmc_boundary_t bnd, double *out,
                        void *workspace, size_t workspace_bytes, wmc_stream_t stream);

/* ------------------------------------------------------------------------------------------
 * Batched denoising: many images of different sizes, each with its own lambda and step, advanced
 * together -- every kernel launch takes T Jacobi steps (wmc_config_t.steps_per_launch, default 4)
 * on the tiles of all images (Sec. V-B flow with A = I; colour channels are images too, as the
 * paper treats them separately, Sec. V-D).
 *
 *   wmc_image_t: f (device, U^0 = f), u (device output), h x w, pitch ld (elements, shared by f
 *   and u), lambda (finite, >= 0), step (finite, > 0).  Images may share f; u must not overlap
 *   any f or any other u.  h or w may be 0 (the image is skipped).
 *
 *   wmc_batch_workspace_size: device bytes for the plan below (status word, per-image
 *   descriptors and tensor maps, the tile table, two ping-pong images per input, and a copy of f
 *   for every input whose f cannot be read through TMA as it is: base or pitch not a multiple of
 *   16 bytes).  The kernels read only 16-byte aligned buffers, whatever the caller's pitch;
 *   u itself is only written, by the last launch of a run.
 *   wmc_batch_plan: validates the images, writes descriptors and the tile table into
 *   `workspace` (device, WMC_WORKSPACE_ALIGN-aligned) and fills `plan` (caller-owned host
 *   memory, opaque).  It synchronises `stream` once, so the `imgs` array may be freed on return.
 *   wmc_batch_run: `iters` Jacobi steps of every image; only kernel launches and one 4-byte
 *   memset are enqueued on `stream` (the first launch refreshes the workspace copies of f, so f
 *   may change between runs), so the call can be captured into a CUDA graph and replayed.
 *   The plan (and its workspace) stays valid until the caller frees them.  wmc_denoise_status()
 *   on the workspace reports a timed-out tile load, as for single images.
 *   wmc_denoise_batched: plan + run in one call.
 * Errors: WMC_ERR_INVALID_ARG (a bad image, count or config; the detail names the image),
 *         WMC_ERR_ALIAS, WMC_ERR_WORKSPACE, WMC_ERR_CUDA.
 */
typedef struct {
    const void *f;
    void *u;
    int32_t h, w;
    int64_t ld;
    float lambda, step;
} wmc_image_t;

typedef struct {
    int64_t opaque[16];
} wmc_batch_t;

size_t wmc_batch_workspace_size(const wmc_image_t *imgs, int32_t n, wmc_dtype_t dtype,
                                const wmc_config_t *config);

wmc_status_t wmc_batch_plan(const wmc_image_t *imgs, int32_t n, wmc_dtype_t dtype,
                            wmc_boundary_t bnd, const wmc_config_t *config, void *workspace,
                            size_t workspace_bytes, wmc_batch_t *plan, wmc_stream_t stream);

wmc_status_t wmc_batch_run(const wmc_batch_t *plan, int32_t iters, wmc_stream_t stream);

wmc_status_t wmc_denoise_batched(const wmc_image_t *imgs, int32_t n, wmc_dtype_t dtype,
                                 int32_t iters, wmc_boundary_t bnd, void *workspace,
                                 size_t workspace_bytes, wmc_stream_t stream);

/*
 * wmc_batch_autotune: picks the steps per launch for a batch by timing it.  For each candidate
 * (NULL = {2, 3, 4, 5, 6, 8}) it plans the batch, runs it once untimed, then runs about
 * trial_iters iterations (rounded up to whole launches) between two CUDA events, and keeps the
 * fastest per iteration.  ms_per_iter (optional, host, n_candidates floats) receives the timings.
 * The trials write the images' outputs (u) and synchronise `stream`; do not capture this call.
 *   workspace: device, >= wmc_batch_autotune_workspace_size() bytes (the largest plan).
 *   best: host, receives {steps_per_launch, tile = 0 (the default shape)} for wmc_batch_plan.
 * Errors: as wmc_batch_plan; WMC_ERR_INVALID_ARG for candidates outside 1..8, n_candidates
 *         outside 1..64 or trial_iters < 1; WMC_ERR_TIMEOUT if a trial reported a timed-out load.
 */
size_t wmc_batch_autotune_workspace_size(const wmc_image_t *imgs, int32_t n, wmc_dtype_t dtype);

/*
 * wmc_batch_autotune_configs: the same search over whole configurations, tile shape included:
 * candidates (host, n_candidates entries of {steps_per_launch 1..8, tile 0..2}; NULL = both tile
 * shapes x steps {2, 3, 4, 5, 6, 8}, 12 candidates in that order, tile-major) are each planned,
 * run once untimed and timed over about trial_iters iterations; `best` receives the fastest
 * candidate as given, ms_per_iter (optional, host) one time per candidate.  The workspace size
 * of wmc_batch_autotune_workspace_size() covers every candidate.  Writes the images' outputs and
 * synchronises `stream`; do not capture this call.
 * Errors: as wmc_batch_autotune; WMC_ERR_INVALID_ARG for a candidate outside those ranges.
 */
wmc_status_t wmc_batch_autotune_configs(const wmc_image_t *imgs, int32_t n, wmc_dtype_t dtype,
                                        wmc_boundary_t bnd, const wmc_config_t *candidates,
                                        int32_t n_candidates, int32_t trial_iters, void *workspace,
                                        size_t workspace_bytes, wmc_config_t *best, float *ms_per_iter,
                                        wmc_stream_t stream);

wmc_status_t wmc_batch_autotune(const wmc_image_t *imgs, int32_t n, wmc_dtype_t dtype,
                                wmc_boundary_t bnd, const int32_t *candidates, int32_t n_candidates,
                                int32_t trial_iters, void *workspace, size_t workspace_bytes,
                                wmc_config_t *best, float *ms_per_iter, wmc_stream_t stream);

/* ------------------------------------------------------------------------------------------
 * The conventional discretisation the paper compares its scheme with (Sec. V-D): Eq. rhs,
 *   H = (U_xx + U_yy) - (U_y^2 U_yy + 2 U_x U_y U_xy + U_x^2 U_xx) / (U_x^2 + U_y^2),
 * with central differences of unit spacing (U_x = (E - W)/2, U_xy = ((SE - NE) - (SW - NW))/4,
 * rows downwards) and H = 0 where the central-difference gradient is exactly zero.
 *   wmc_eval_fd: as wmc_eval, with this H.
 *   wmc_denoise_fd: as wmc_denoise (f NULL = mean-curvature flow), with this H and one streaming
 *   launch per iteration; workspace as wmc_denoise_workspace_size().
 * Errors: as wmc_eval / wmc_denoise.
 */
wmc_status_t wmc_eval_fd(const void *u, void *hw, int32_t h, int32_t w, int64_t ld_u,
                         int64_t ld_hw, wmc_dtype_t dtype, wmc_boundary_t bnd,
                         wmc_stream_t stream);

wmc_status_t wmc_denoise_fd(const void *f, const void *u0, void *u, int32_t h, int32_t w, int64_t ld,
                            wmc_dtype_t dtype, float lambda, float step, int32_t iters,
                            wmc_boundary_t bnd, void *workspace, size_t workspace_bytes,
                            wmc_stream_t stream);

/* ------------------------------------------------------------------------------------------
 * wmc_denoise_l1: the L1-fidelity model min_U ||U - f||_1 + lambda R(U) solved by the primal-dual
 * iteration of Sec. V-C with A = I (b eliminated):
 *   r = U^t - f + d^t;  d^{t+1} = clip(r, -alpha, alpha);
 *   U^{t+1} = U^t + step * (lambda H^w(U^t) - (2 d^{t+1} - d^t) / alpha)      t = 0..iters-1
 * The paper gives neither alpha nor step; both are arguments (alpha > 0 "small").
 *   f: device FP32, h x w, pitch ld.  u0: U^0 (device; NULL = f; may equal u for resuming in
 *   place).  u: output U^iters.  d: the scaled dual variable, device FP32 with pitch ld, read as
 *   d^0 and overwritten with d^iters; NULL = start from d^0 = 0 and discard it.
 *   workspace: device, >= wmc_denoise_l1_workspace_size() bytes (status word, one ping-pong
 *   image, one d image), aligned to WMC_WORKSPACE_ALIGN.  One kernel launch per iteration.
 * Errors: WMC_ERR_INVALID_ARG (sizes, lambda < 0, step <= 0, alpha <= 0, non-finite values,
 *         iters < 0, NULL f or u), WMC_ERR_ALIAS (u overlaps f or, unless equal, u0; d overlaps
 *         f, u or u0; workspace overlaps an image), WMC_ERR_WORKSPACE, WMC_ERR_CUDA.
 */
size_t wmc_denoise_l1_workspace_size(int32_t h, int32_t w, int64_t ld);

wmc_status_t wmc_denoise_l1(const float *f, const float *u0, float *u, float *d, int32_t h, int32_t w,
                            int64_t ld, float lambda, float step, float alpha, int32_t iters,
                            wmc_boundary_t bnd, void *workspace, size_t workspace_bytes,
                            wmc_stream_t stream);

/* ------------------------------------------------------------------------------------------
 * Reverse mode (training through the flow).  The paper uses H^w as a descent direction and
 * leaves the gradient of its regulariser open (Sec. III after Eq. wmcr); H^w is piecewise linear
 * in U, and on the piece picked by the selection of Eq. act it is the correlation of U with the
 * selected kernel h_m (Sec. IV-B).  These calls differentiate with each pixel's selection held at
 * its forward value (a subgradient where the selection switches).  FP32 only.
 *
 * Unrolled denoising of a stack of n equally sized images (image i at f + i*h*ld elements):
 *   U^0 = f,  U^{t+1} = U^t + step*(lambda_i H^w(U^t) - (U^t - f))   t = 0..K-1
 * (the Sec. V-B flow with A = I, Jacobi; bitwise the same values as wmc_denoise on each image).
 *   lambda: DEVICE, n floats (one per image, read by the kernels, so it may change between
 *   graph replays).  step: > 0, shared.  K >= 0 steps.  ckpt_every >= 1: the forward keeps
 *   U^c, U^2c, ... in the workspace and the backward recomputes the steps between checkpoints
 *   (memory ~ (K/c + c) images instead of K).
 *   wmc_unrolled_workspace_size: device bytes for both calls (0 for invalid sizes).
 *   wmc_unrolled_forward: u (device, n x h x ld) = U^K.  The workspace then holds the
 *   checkpoints that wmc_unrolled_backward reads: pass the same workspace, f, lambda, step, K,
 *   ckpt_every and sizes, with no other call on that workspace in between.
 *   wmc_unrolled_backward: given grad_u = dL/dU^K (device, n x h x ld), writes
 *   grad_f = dL/df (device, n x h x ld) and grad_lambda = dL/dlambda (device, n floats).
 *   The lambda sums run in FP64 in a fixed order (reproducible).
 * Errors: WMC_ERR_INVALID_ARG (sizes, n outside 1..65535, K < 0, ckpt_every < 1, step <= 0,
 *         NULL pointers), WMC_ERR_ALIAS (u overlaps f; grad_f overlaps grad_u or f; workspace
 *         overlaps an image), WMC_ERR_WORKSPACE (too small or misaligned), WMC_ERR_CUDA.
 */
size_t wmc_unrolled_workspace_size(int32_t n, int32_t h, int32_t w, int64_t ld, int32_t K,
                                   int32_t ckpt_every);

wmc_status_t wmc_unrolled_forward(const float *f, const float *lambda, float step, int32_t K,
                                  int32_t ckpt_every, int32_t n, int32_t h, int32_t w, int64_t ld,
                                  wmc_boundary_t bnd, float *u, void *workspace,
                                  size_t workspace_bytes, wmc_stream_t stream);

wmc_status_t wmc_unrolled_backward(const float *f, const float *lambda, float step, int32_t K,
                                   int32_t ckpt_every, int32_t n, int32_t h, int32_t w, int64_t ld,
                                   wmc_boundary_t bnd, const float *grad_u, float *grad_f,
                                   float *grad_lambda, void *workspace, size_t workspace_bytes,
                                   wmc_stream_t stream);

/*
 * wmc_backward: the reverse mode of K unrolled denoising steps in one call, with the arguments
 * of the problem statement: f (device, n x h x ld stack), lambda (device, n floats), step, K,
 * ckpt_every, and grad_u = dL/dU^K (device, n x h x ld) in; grad_f = dL/df (device, n x h x ld)
 * and grad_lambda = dL/dlambda (device, n floats) out.  It runs wmc_unrolled_forward (keeping
 * U^K and the checkpoints in the workspace) and then wmc_unrolled_backward; use those two calls
 * instead when U^K itself is wanted, so that the forward is not run twice.  Selection held at its
 * forward value, as above.
 *   workspace: device, >= wmc_backward_workspace_size() bytes (the unrolled workspace plus one
 *   stack for U^K), WMC_WORKSPACE_ALIGN-aligned, overlapping none of f, grad_u, grad_f.
 * Errors: as wmc_unrolled_backward.
 */
size_t wmc_backward_workspace_size(int32_t n, int32_t h, int32_t w, int64_t ld, int32_t K,
                                   int32_t ckpt_every);

wmc_status_t wmc_backward(const float *f, const float *lambda, float step, int32_t K,
                          int32_t ckpt_every, int32_t n, int32_t h, int32_t w, int64_t ld,
                          wmc_boundary_t bnd, const float *grad_u, float *grad_f,
                          float *grad_lambda, void *workspace, size_t workspace_bytes,
                          wmc_stream_t stream);

/*
 * wmc_energy_grad: grad = d/dU sum_p |H^w(U)(p)| (the Eq. wmcr regulariser, q = 1), selection
 * held fixed, sign(0) = 0.  u, grad: device FP32, h x w, pitch ld, must not overlap.  One kernel
 * launch, no workspace.
 */
wmc_status_t wmc_energy_grad(const float *u, float *grad, int32_t h, int32_t w, int64_t ld,
                             wmc_boundary_t bnd, wmc_stream_t stream);

/* ------------------------------------------------------------------------------------------
 * wmc_shard_lpt: host-side partition of n independent images over `world` ranks (one GPU each),
 * for running a batch of Sec. V-B denoisings on several GPUs with no communication: each image
 * goes to one rank, balancing the ranks' total cost (cost[i]: the image's pixel count, or pixels
 * x iterations).  Longest-processing-time-first (Graham): images in order of decreasing cost
 * (equal costs: lower index first), each to the rank with the least cost so far (equal loads:
 * lower rank).  The largest load is at most (4/3 - 1/(3 world)) of the best possible.  The
 * result depends only on the arguments, so every rank computes the same partition by itself.
 *   cost: host, n entries >= 0.  owner: host, n entries, written (rank of image i).
 *   load: host, `world` entries, written (each rank's total cost), or NULL.
 *   n >= 0 (0: nothing to do), world >= 1; cost and owner non-NULL when n > 0.
 *   Runs on the calling thread, no CUDA call; WMC_ERR_INVALID_ARG on bad arguments.
 */
wmc_status_t wmc_shard_lpt(const int64_t *cost, int32_t n, int32_t world, int32_t *owner,
                           int64_t *load);

/* ------------------------------------------------------------------------------------------
 * wmc_probe_fma: a measurement utility with no counterpart in the paper.  Enqueues `blocks` CTAs
 * of wmc_probe_fma_threads() threads, each thread running `iters` iterations of 16 FP32 fused
 * multiply-adds (8 independent packed FP32x2 chains), and writing one float per thread to `out`
 * (device, blocks * wmc_probe_fma_threads() floats).  Timing it with events gives the FP32 FMA
 * pipe's rate in lane-operations per second (an FMA counts once): the compute roofline of the
 * temporally blocked flow kernel.  blocks 1 .. 2^20, iters >= 1.
 * Errors: WMC_ERR_INVALID_ARG, WMC_ERR_CUDA (launch failure).
 */
int32_t wmc_probe_fma_threads(void);
wmc_status_t wmc_probe_fma(float *out, int32_t blocks, int32_t iters, wmc_stream_t stream);

/* ------------------------------------------------------------------------------------------ */
const char *wmc_status_string(wmc_status_t status); /* static string, never NULL */
const char *wmc_last_error(void); /* detail of the last failure on this thread ("" if none) */
int32_t wmc_version(void);        /* 100 * major + minor */

#ifdef __cplusplus
}
#endif

#endif /* WMC_H */
