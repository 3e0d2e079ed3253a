// wmc_api.cu -- the C ABI declared in include/wmc.h: argument checks, workspace layout and
// the host-side loop that drives the stencil kernels on the caller's stream.
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>

#include <algorithm>
#include <atomic>
#include <mutex>
#include <vector>

#include <cuda.h>
#include <cudaTypedefs.h>
#include <cuda_runtime.h>

#include "../../include/wmc.h"
#include "wmc_internal.h"
#include "wmc_stream.cuh"
#include "wmc_tile.cuh"

namespace wmc {
void tile_box(int dtype, int tile, int *bw, int *bh) {
    *bw = dtype == 0 ? Geom<float>::LW : Geom<__half>::LW;
    *bh = kQR * tile_warps(tile) + 2;
}
}  // namespace wmc

namespace {

thread_local char g_last_error[512] = "";

wmc_status_t fail(wmc_status_t s, const char *fmt, ...) {
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(g_last_error, sizeof g_last_error, fmt, ap);
    va_end(ap);
    return s;
}

wmc_status_t cuda_fail(cudaError_t e, const char *what) {
    return fail(WMC_ERR_CUDA, "%s: %s (%s)", what, cudaGetErrorName(e), cudaGetErrorString(e));
}

size_t elem_size(wmc_dtype_t t) {
    switch (t) {
        case WMC_F32: return 4;
        case WMC_BF16:
        case WMC_F16: return 2;
        default: return 0;
    }
}

// Bytes spanned by an h x w image with pitch ld.
size_t span_bytes(int32_t h, int32_t w, int64_t ld, size_t es) {
    if (h <= 0 || w <= 0) return 0;
    return ((size_t)(h - 1) * (size_t)ld + (size_t)w) * es;
}

bool overlap(const void *a, size_t na, const void *b, size_t nb) {
    if (!a || !b || na == 0 || nb == 0) return false;
    const uintptr_t pa = (uintptr_t)a, pb = (uintptr_t)b;
    return pa < pb + nb && pb < pa + na;
}

size_t round_up(size_t v, size_t a) { return (v + a - 1) / a * a; }

constexpr int32_t kMaxSide = 1 << 24;

wmc_status_t check_image(int32_t h, int32_t w, int64_t ld, const char *name) {
    if (h < 0 || w < 0) return fail(WMC_ERR_INVALID_ARG, "%s: negative size %d x %d", name, h, w);
    if (h > 0 && w > 0 && ld < w)
        return fail(WMC_ERR_INVALID_ARG, "%s: leading dimension %lld < width %d", name,
                    (long long)ld, w);
    if (h > kMaxSide || w > kMaxSide)
        return fail(WMC_ERR_INVALID_ARG, "%s: side longer than %d", name, kMaxSide);
    return WMC_OK;
}

wmc_status_t check_enums(wmc_dtype_t dtype, wmc_boundary_t bnd) {
    if (elem_size(dtype) == 0) return fail(WMC_ERR_INVALID_ARG, "unknown dtype %d", (int)dtype);
    if (bnd != WMC_BOUNDARY_REPLICATE && bnd != WMC_BOUNDARY_ZERO)
        return fail(WMC_ERR_INVALID_ARG, "unknown boundary %d", (int)bnd);
    return WMC_OK;
}

// ------------------------------------------------------------------ TMA descriptors
PFN_cuTensorMapEncodeTiled_v12000 g_encode = nullptr;
std::once_flag g_encode_once;

PFN_cuTensorMapEncodeTiled_v12000 encoder() {
    std::call_once(g_encode_once, [] {
        void *fn = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault,
                                             &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            g_encode = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(fn);
        else
            cudaGetLastError();
    });
    return g_encode;
}

// A 2-D tiled tensor map over an h x w image with pitch ld and a bw x bh box.  Returns false
// when the image cannot be read through TMA (alignment, pitch, driver).
bool encode_box_map(CUtensorMap *m, const void *base, wmc_dtype_t dtype, int32_t h, int32_t w,
                    int64_t ld, int bw, int bh) {
    const size_t es = elem_size(dtype);
    if (((uintptr_t)base % 16) != 0 || ((size_t)ld * es) % 16 != 0) return false;
    if ((size_t)ld * es >= (1ull << 40)) return false;
    PFN_cuTensorMapEncodeTiled_v12000 enc = encoder();
    if (!enc) return false;
    const CUtensorMapDataType t = dtype == WMC_F32    ? CU_TENSOR_MAP_DATA_TYPE_FLOAT32
                                  : dtype == WMC_BF16 ? CU_TENSOR_MAP_DATA_TYPE_BFLOAT16
                                                      : CU_TENSOR_MAP_DATA_TYPE_FLOAT16;
    cuuint64_t dims[2] = {(cuuint64_t)w, (cuuint64_t)h};
    cuuint64_t strides[1] = {(cuuint64_t)ld * es};
    cuuint32_t box[2] = {(cuuint32_t)bw, (cuuint32_t)bh};
    cuuint32_t estr[2] = {1, 1};
    const CUresult r = enc(m, t, 2, const_cast<void *>(base), dims, strides, box, estr,
                           CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                           CU_TENSOR_MAP_L2_PROMOTION_L2_128B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    return r == CUDA_SUCCESS;
}

// The same with the window of the flow kernel's tile shape `tile` as the box (tile 1: the 136 x 66
// window of a 128 x 64 box, which the evaluation and energy kernels load too).
bool encode_window_map(CUtensorMap *m, const void *base, wmc_dtype_t dtype, int32_t h, int32_t w,
                       int64_t ld, int tile = 1) {
    int bw, bh;
    wmc::tile_box((int)dtype, tile, &bw, &bh);
    return encode_box_map(m, base, dtype, h, w, ld, bw, bh);
}

bool pair_aligned(const void *p, int64_t ld, size_t es) {
    return p == nullptr || (((uintptr_t)p % (2 * es)) == 0 && (ld % 2) == 0);
}

// batch_tiles < 0: single-image launch (tiles from the grid); >= 0: batch launch over that
// many tiles of the plan's table.
cudaError_t launch_tile(wmc_dtype_t dtype, wmc_boundary_t bnd, int tile, int steps, const CUtensorMap *map,
                        const wmc::TileParams &p, int64_t batch_tiles, cudaStream_t st) {
    const bool z = bnd == WMC_BOUNDARY_ZERO, s = tile == 2;
#define WMC_TILE_PICK(dt)                                                                         \
    (z ? (s ? wmc::launch_tile_##dt##_zero_w8 : wmc::launch_tile_##dt##_zero_w16)                 \
       : (s ? wmc::launch_tile_##dt##_rep_w8 : wmc::launch_tile_##dt##_rep_w16))
    switch (dtype) {
        case WMC_F32: return WMC_TILE_PICK(f32)(steps, map, p, batch_tiles, st);
        case WMC_BF16: return WMC_TILE_PICK(bf16)(steps, map, p, batch_tiles, st);
        case WMC_F16: return WMC_TILE_PICK(f16)(steps, map, p, batch_tiles, st);
        default: return cudaErrorInvalidValue;
    }
#undef WMC_TILE_PICK
}

constexpr int kDefaultTile = 1;
constexpr int kTileShapes = 2;  // wmc_config_t.tile = 1 .. kTileShapes (0: kDefaultTile)

constexpr int kDefaultSteps = 4;
// Fewest iterations for which the default configuration runs a small image as one cluster launch
constexpr int kClusterMinIters = 2;
constexpr size_t kStatusBytes = WMC_WORKSPACE_ALIGN;

size_t image_bytes(int32_t h, int64_t ld, wmc_dtype_t dtype) {
    return round_up((size_t)h * (size_t)ld * elem_size(dtype), WMC_WORKSPACE_ALIGN);
}

// Whether an image with this pitch is staged through aligned workspace images for the
// temporally blocked launches (TMA reads need a pitch that is a multiple of 16 bytes).
bool staged_pitch(int64_t ld, size_t es) { return ((size_t)ld * es) % 16 != 0; }

int64_t aligned_pitch(int32_t w, size_t es) {
    const int64_t A = 16 / (int64_t)es;
    return (w + A - 1) / A * A;
}

// Output tile of T steps per launch with tile shape `tile`: the region less T - 1 cells (plus the
// region's own halo) on each side.
void out_tile(int T, int tile, int *owt, int *oht) {
    *owt = wmc::kCW + 2 - 2 * T;
    *oht = wmc::kQR * wmc::tile_warps(tile) + 2 - 2 * T;
}

// Launches of more waves of CTAs than this wait for the whole previous launch (see run_flow).
constexpr int kFlagMaxWaves = 10;

// Per-tile completion flags of a flow run: one word per tile of the largest tile grid any
// multi-step launch of an h x w image can have (8 steps per launch, the 128 x 32 region).
int64_t flow_flag_words(int32_t h, int32_t w) {
    int64_t most = 0;
    for (int tile = 1; tile <= kTileShapes; ++tile)
        for (int T = 2; T <= wmc::kMaxSteps; ++T) {
            int owt, oht;
            out_tile(T, tile, &owt, &oht);
            most = std::max(most, (int64_t)((w + owt - 1) / owt) * ((h + oht - 1) / oht));
        }
    return most;
}

// Workspace of run_flow without the flags: the status word (first kStatusBytes) followed by one
// image of pitch ld, or, for pitches TMA cannot describe, three images of an aligned pitch (two
// ping-pong images and a copy of f), and at least one image of pitch ld for the calls that are
// not staged (one launch, or one step per launch).
size_t flow_core_bytes(int32_t h, int32_t w, int64_t ld, wmc_dtype_t dtype) {
    const size_t es = elem_size(dtype);
    if (staged_pitch(ld, es))
        return std::max(3 * image_bytes(h, aligned_pitch(w, es), dtype), image_bytes(h, ld, dtype)) + kStatusBytes;
    return image_bytes(h, ld, dtype) + kStatusBytes;
}

// The flow on device buffers; all checks done by the caller.  `ws` holds what flow_core_bytes
// counts, so that every buffer a multi-step launch reads is TMA-readable and only the last launch
// touches u.  `flags` (flow_flag_words words, or nullptr): the tiles of consecutive launches with
// the same tile grid then wait only for the tiles of the previous launch they depend on, instead
// of for that whole launch.
wmc_status_t run_flow(const void *f, const void *u0, void *u, int32_t h, int32_t w, int64_t ld,
                      wmc_dtype_t dtype, float lambda, float step, int32_t iters,
                      wmc_boundary_t bnd, int steps_per_launch, void *ws, cudaStream_t st,
                      bool fd = false, int tile = kDefaultTile, bool default_config = false,
                      unsigned int *flags = nullptr) {
    const size_t es = elem_size(dtype);
    if (!u0) u0 = f;
    if (h == 0 || w == 0) return WMC_OK;
    if (iters == 0) {
        if (u0 != u) {
            cudaError_t e = cudaMemcpy2DAsync(u, ld * es, u0, ld * es, w * es, h,
                                              cudaMemcpyDeviceToDevice, st);
            if (e != cudaSuccess) return cuda_fail(e, "copy U^0");
        }
        return WMC_OK;
    }
    unsigned int *status = static_cast<unsigned int *>(ws);
    ws = static_cast<char *>(ws) + kStatusBytes;
    const float mu = f ? 1.0f : 0.0f;
    const float c_keep = 1.0f - step * mu, c_f = step * mu;
    const float c_h = fd ? step * lambda : step * lambda / 12.0f;
    cudaError_t e;
    // Small images under the default configuration: all the iterations in one cluster launch
    // (it clears the status word itself and needs no workspace image)
    if (!fd && default_config && iters >= kClusterMinIters) {
        const int ctas = wmc::cluster_ctas(h, w);
        if (ctas > 0 && wmc::cluster_fits(ctas)) {
            e = wmc::launch_flow_cluster((int)dtype, (int)bnd, u0, f, u, status, ld, ld, h, w, iters, c_keep,
                                         c_f, c_h, st);
            return e == cudaSuccess ? WMC_OK : cuda_fail(e, "cluster flow kernel launch");
        }
    }
    e = cudaMemsetAsync(status, 0, sizeof(unsigned int), st);
    if (e != cudaSuccess) return cuda_fail(e, "clear status");

    const int T = fd ? 1 : steps_per_launch;  // the finite-difference comparator streams
    const int nl = (iters + T - 1) / T;  // launches; the last takes the remainder
    // Buffers: launch k reads src_k (pitch ld_in) and writes dst_k (pitch ld_out on the last
    // launch, ld_in otherwise); f_read is the f the launches read.
    const bool staged = T > 1 && nl > 1 && staged_pitch(ld, es);
    const int64_t ld_in = staged ? aligned_pitch(w, es) : ld;
    const void *f_read = f;
    void *bufs[2];
    bool copy_back = false;
    const void *src = u0;
    if (staged) {
        // U^0 and f copied into aligned images; the launches between the first and the last
        // ping-pong between the two ping-pong images
        const size_t one = image_bytes(h, ld_in, dtype);
        char *A = static_cast<char *>(ws), *B = A + one, *F = B + one;
        e = cudaMemcpy2DAsync(A, ld_in * es, u0, ld * es, w * es, h, cudaMemcpyDeviceToDevice, st);
        if (e == cudaSuccess && f)
            e = cudaMemcpy2DAsync(F, ld_in * es, f, ld * es, w * es, h, cudaMemcpyDeviceToDevice, st);
        if (e != cudaSuccess) return cuda_fail(e, "stage U^0 and f");
        src = A;
        f_read = f ? F : nullptr;
        bufs[0] = B;
        bufs[1] = A;
    } else if (u0 == u) {
        // Ping-pong between u and the workspace so that the last launch writes u.  When U^0
        // already lives in u, the first launch must write the workspace; if the parity then
        // ends in the workspace, one copy finishes the job.
        bufs[0] = ws;
        bufs[1] = u;
        copy_back = (nl % 2) == 1;
    } else if (nl % 2 == 1) {
        bufs[0] = u;
        bufs[1] = ws;
    } else {
        bufs[0] = ws;
        bufs[1] = u;
    }
    const bool vec = pair_aligned(src, ld_in, es) && pair_aligned(f_read, ld_in, es) &&
                     pair_aligned(u, ld, es) && pair_aligned(bufs[0], ld_in, es) && pair_aligned(bufs[1], ld_in, es);
    // Tensor maps for every buffer a tile launch may read: U^0 and the two ping-pong buffers.
    CUtensorMap maps[3];
    bool tma[3] = {false, false, false};
    const void *srcs[3] = {src, bufs[0], bufs[1]};
    if (T > 1)
        for (int k = 0; k < 3; ++k) tma[k] = encode_window_map(&maps[k], srcs[k], dtype, h, w, ld_in, tile);
    // f's window is loaded by TMA with U's (same box)
    alignas(64) CUtensorMap fmap;
    memset(&fmap, 0, sizeof fmap);
    const bool f_tma = T > 1 && f_read != nullptr && encode_window_map(&fmap, f_read, dtype, h, w, ld_in, tile);

    // the flags start at 0 in every run; launch number e (1, 2, ...) stores e into each of its
    // tiles'.  They cost each tile a memory round trip before its load and a release after its
    // stores (about 5 % of a launch on its own), and save the previous launch's last wave, which
    // the wait for that whole launch leaves partly idle: a gain for launches of a few waves of
    // CTAs (2 per SM), a loss for one wave or less (a launch's tiles then depend on most of the
    // previous launch anyway) and for many waves (the last wave is then a small part).
    if (T == 1 || nl == 1) flags = nullptr;
    if (flags) {
        int owt, oht, dev = 0, nsm = 0;
        out_tile(T, tile, &owt, &oht);
        const int64_t ntiles = (int64_t)((w + owt - 1) / owt) * ((h + oht - 1) / oht);
        e = cudaGetDevice(&dev);
        if (e == cudaSuccess) e = cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
        if (e != cudaSuccess) return cuda_fail(e, "query the SM count");
        if (ntiles <= 2 * (int64_t)nsm || ntiles > kFlagMaxWaves * 2 * (int64_t)nsm) flags = nullptr;
    }
    if (flags) {
        e = cudaMemsetAsync(flags, 0, (size_t)flow_flag_words(h, w) * sizeof(unsigned int), st);
        if (e != cudaSuccess) return cuda_fail(e, "clear tile flags");
    }
    int src_id = 0;
    int done = 0;
    bool prev_tile = false;
    int prev_s = 0, epoch = 0;
    for (int k = 0; k < nl; ++k) {
        const int s = (iters - done) < T ? (iters - done) : T;
        const bool last = k == nl - 1;
        void *dst = (staged && last) ? u : bufs[k & 1];
        const int64_t ldo = (staged && last) ? ld : ld_in;
        if (s == 1) {
            wmc::StreamParams sp{};
            sp.u = src;
            sp.f = f_read;
            sp.out = dst;
            sp.ldu = sp.ldf = ld_in;
            sp.ldo = ldo;
            sp.h = h;
            sp.w = w;
            sp.c_keep = c_keep;
            sp.c_f = c_f;
            sp.c_h = c_h;
            e = wmc::launch_stream((int)dtype, fd ? wmc::MODE_FD_FLOW : wmc::MODE_FLOW, (int)bnd, sp,
                                   vec, st);
        } else {
            wmc::TileParams tp{};
            tp.u = src;
            tp.f = f_read;
            tp.out = dst;
            tp.ld = ld_in;
            tp.ld_out = ldo;
            tp.h = h;
            tp.w = w;
            tp.use_tma = tma[src_id] ? 1 : 0;
            tp.c_keep = c_keep;
            tp.c_f = c_f;
            tp.c_h = c_h;
            tp.status = status;
            tp.pdl = prev_tile ? 1 : 0;  // follows a tile launch: may overlap its tail
            tp.f_tma = (f_tma && tma[src_id]) ? 1 : 0;
            if (flags) {
                // the previous launch has the same tile grid: wait for its tiles, not for all of it
                tp.flags = flags;
                tp.flag_wait = (prev_tile && prev_s == s && tma[src_id]) ? epoch : 0;
                tp.flag_set = ++epoch;
            }
            alignas(64) CUtensorMap pair[2] = {maps[src_id], fmap};
            e = launch_tile(dtype, bnd, tile, s, pair, tp, -1, st);
        }
        if (e != cudaSuccess) return cuda_fail(e, "flow kernel launch");
        prev_tile = s > 1;
        prev_s = s;
        src = dst;
        src_id = 1 + (k & 1);
        done += s;
    }
    if (copy_back) {
        e = cudaMemcpy2DAsync(u, ld * es, src, ld * es, w * es, h, cudaMemcpyDeviceToDevice, st);
        if (e != cudaSuccess) return cuda_fail(e, "copy result");
    }
    return WMC_OK;
}

wmc_status_t check_flow_args(const void *f, const void *u0, void *u, int32_t h, int32_t w,
                             int64_t ld, wmc_dtype_t dtype, float lambda, float step,
                             int32_t iters, wmc_boundary_t bnd, const wmc_config_t *cfg,
                             int *steps_out, int *tile_out = nullptr, bool *default_out = nullptr) {
    wmc_status_t s;
    if ((s = check_enums(dtype, bnd)) != WMC_OK) return s;
    if ((s = check_image(h, w, ld, "image")) != WMC_OK) return s;
    if (!std::isfinite(lambda) || lambda < 0.0f)
        return fail(WMC_ERR_INVALID_ARG, "lambda must be finite and >= 0 (got %g)", lambda);
    if (!std::isfinite(step) || step <= 0.0f)
        return fail(WMC_ERR_INVALID_ARG, "step must be finite and > 0 (got %g)", step);
    if (iters < 0) return fail(WMC_ERR_INVALID_ARG, "iters must be >= 0 (got %d)", iters);
    int T = kDefaultSteps;
    if (cfg) {
        if (cfg->steps_per_launch < 0 || cfg->steps_per_launch > wmc::kMaxSteps)
            return fail(WMC_ERR_INVALID_ARG, "steps_per_launch must be 0..%d (got %d)",
                        wmc::kMaxSteps, cfg->steps_per_launch);
        if (cfg->tile < 0 || cfg->tile > kTileShapes)
            return fail(WMC_ERR_INVALID_ARG, "unknown tile %d (0 .. %d)", cfg->tile, kTileShapes);
        if (cfg->steps_per_launch > 0) T = cfg->steps_per_launch;
    }
    *steps_out = T;
    if (tile_out) *tile_out = (cfg && cfg->tile > 0) ? cfg->tile : kDefaultTile;
    if (default_out) *default_out = !cfg || (cfg->steps_per_launch == 0 && cfg->tile == 0);
    if (h > 0 && w > 0) {
        if (!u) return fail(WMC_ERR_INVALID_ARG, "u is NULL");
        if (!f && !u0) return fail(WMC_ERR_INVALID_ARG, "f and u0 are both NULL");
        const size_t n = span_bytes(h, w, ld, elem_size(dtype));
        if (overlap(u, n, f, n)) return fail(WMC_ERR_ALIAS, "u overlaps f");
        if (u0 && u0 != u && overlap(u, n, u0, n)) return fail(WMC_ERR_ALIAS, "u overlaps u0");
    }
    return WMC_OK;
}

// ------------------------------------------------------------------ batches
constexpr uint32_t kBatchMagic = 0x57424348u;  // "WBCH"

struct BatchPlan {
    void *ws;
    int64_t ntiles;
    int64_t off_images, off_tiles;
    int32_t n, dtype, bnd, steps;
    int32_t owt, oht;
    int32_t tile;
    int32_t any_copy;  // some image reads a workspace copy of its f
    uint32_t magic;
};
static_assert(sizeof(BatchPlan) <= sizeof(wmc_batch_t), "plan does not fit wmc_batch_t");

struct BatchLayout {
    size_t off_images, off_tiles, off_bufs, total;
    int64_t ntiles;
    std::vector<size_t> buf_off;   // per image: two ping-pong images, then f's copy if needed
    std::vector<int64_t> ld_read;  // per image: pitch of the buffers the kernels read
    std::vector<char> copy_f;      // per image: f is copied into the workspace (pitch or base not TMA-able)
};

// The caller's buffer can be read through TMA as it is: 16-byte aligned base and pitch.
bool tma_able(const void *p, int64_t ld, size_t es) {
    return ((uintptr_t)p % 16) == 0 && ((size_t)ld * es) % 16 == 0;
}

BatchLayout batch_layout(const wmc_image_t *imgs, int32_t n, wmc_dtype_t dtype, int T, int tile) {
    BatchLayout L{};
    int owt, oht;
    out_tile(T, tile, &owt, &oht);
    L.off_images = kStatusBytes;
    L.off_tiles = round_up(L.off_images + (size_t)n * sizeof(wmc::BatchImage), WMC_WORKSPACE_ALIGN);
    L.ntiles = 0;
    for (int32_t i = 0; i < n; ++i)
        if (imgs[i].h > 0 && imgs[i].w > 0)
            L.ntiles += (int64_t)((imgs[i].w + owt - 1) / owt) * ((imgs[i].h + oht - 1) / oht);
    L.off_bufs = round_up(L.off_tiles + (size_t)L.ntiles * sizeof(int4), WMC_WORKSPACE_ALIGN);
    size_t off = L.off_bufs;
    const size_t es = elem_size(dtype);
    const int64_t A = 16 / (int64_t)es;
    L.buf_off.resize(n);
    L.ld_read.resize(n);
    L.copy_f.resize(n);
    for (int32_t i = 0; i < n; ++i) {
        L.buf_off[i] = off;
        const wmc_image_t &m = imgs[i];
        const bool copy = !tma_able(m.f, m.ld, es);
        L.copy_f[i] = copy;
        L.ld_read[i] = copy ? (m.w + A - 1) / A * A : m.ld;
        if (m.h > 0 && m.w > 0) off += (copy ? 3 : 2) * image_bytes(m.h, L.ld_read[i], dtype);
    }
    L.total = off;
    return L;
}

int batch_steps(const wmc_config_t *cfg) {
    return (cfg && cfg->steps_per_launch > 0) ? cfg->steps_per_launch : kDefaultSteps;
}

int batch_tile(const wmc_config_t *cfg) { return (cfg && cfg->tile > 0) ? cfg->tile : kDefaultTile; }

wmc_status_t check_batch(const wmc_image_t *imgs, int32_t n, wmc_dtype_t dtype, wmc_boundary_t bnd,
                         const wmc_config_t *cfg) {
    wmc_status_t s;
    if ((s = check_enums(dtype, bnd)) != WMC_OK) return s;
    if (n < 0) return fail(WMC_ERR_INVALID_ARG, "negative image count %d", n);
    if (n > 0 && !imgs) return fail(WMC_ERR_INVALID_ARG, "imgs is NULL");
    if (cfg) {
        if (cfg->steps_per_launch < 0 || cfg->steps_per_launch > wmc::kMaxSteps)
            return fail(WMC_ERR_INVALID_ARG, "steps_per_launch must be 0..%d (got %d)",
                        wmc::kMaxSteps, cfg->steps_per_launch);
        if (cfg->tile < 0 || cfg->tile > kTileShapes)
            return fail(WMC_ERR_INVALID_ARG, "unknown tile %d (0 .. %d)", cfg->tile, kTileShapes);
    }
    const size_t es = elem_size(dtype);
    // every u must be disjoint from every other buffer; f buffers may overlap each other
    struct Iv { uintptr_t a, b; bool is_u; int32_t img; };
    std::vector<Iv> iv;
    iv.reserve(2 * (size_t)n);
    for (int32_t i = 0; i < n; ++i) {
        const wmc_image_t &m = imgs[i];
        if (m.h < 0 || m.w < 0)
            return fail(WMC_ERR_INVALID_ARG, "image %d: negative size %d x %d", i, m.h, m.w);
        if (m.h > kMaxSide || m.w > kMaxSide)
            return fail(WMC_ERR_INVALID_ARG, "image %d: side longer than %d", i, kMaxSide);
        if (m.h == 0 || m.w == 0) continue;
        if (m.ld < m.w)
            return fail(WMC_ERR_INVALID_ARG, "image %d: leading dimension %lld < width %d", i,
                        (long long)m.ld, m.w);
        if (!m.f || !m.u) return fail(WMC_ERR_INVALID_ARG, "image %d: NULL f or u", i);
        if (!std::isfinite(m.lambda) || m.lambda < 0.0f)
            return fail(WMC_ERR_INVALID_ARG, "image %d: lambda must be finite and >= 0", i);
        if (!std::isfinite(m.step) || m.step <= 0.0f)
            return fail(WMC_ERR_INVALID_ARG, "image %d: step must be finite and > 0", i);
        const size_t nb = span_bytes(m.h, m.w, m.ld, es);
        iv.push_back({(uintptr_t)m.f, (uintptr_t)m.f + nb, false, i});
        iv.push_back({(uintptr_t)m.u, (uintptr_t)m.u + nb, true, i});
    }
    std::sort(iv.begin(), iv.end(), [](const Iv &x, const Iv &y) {
        return x.a < y.a || (x.a == y.a && x.b < y.b);
    });
    uintptr_t maxend = 0;
    const Iv *holder = nullptr;
    for (const Iv &x : iv) {
        if (holder && x.a < maxend && (x.is_u || holder->is_u))
            return fail(WMC_ERR_ALIAS, "image %d: output overlaps image %d", x.is_u ? x.img : holder->img,
                        x.is_u ? holder->img : x.img);
        if (x.b > maxend) {
            maxend = x.b;
            holder = &x;
        }
    }
    return WMC_OK;
}

// Copies the caller's f of every output tile: into u (to_u: a run with zero iterations), or
// into the workspace copy the kernels read, for the images that have one (at the start of a run).
template <typename E>
__global__ void batch_copy_kernel(const wmc::BatchImage *images, const int4 *tiles, int owt, int oht, int to_u) {
    const int4 t = tiles[blockIdx.x];
    const wmc::BatchImage &im = images[t.x];
    if (!to_u && !im.copy_f) return;
    const E *f = static_cast<const E *>(im.f_src);
    E *dst = static_cast<E *>(const_cast<void *>(im.buf[to_u ? 1 : 0]));
    const int64_t ldd = to_u ? im.ld_out : im.ld;
    for (int idx = threadIdx.x; idx < owt * oht; idx += blockDim.x) {
        const int y = t.z + idx / owt, x = t.y + idx % owt;
        if (y < im.h && x < im.w) dst[(int64_t)y * ldd + x] = f[(int64_t)y * im.ld_out + x];
    }
}

// Unrolled-flow workspace: [256 reserved bytes (the status-word slot of the other workspaces;
// these kernels have no bounded waits) | checkpoints | segment/temporary stacks | g ping-pong |
// dlambda partials].
struct UnrolledLayout {
    size_t slot, off_ckpt, off_seg, off_g, off_part, total;
    int32_t ncp, nseg;
    int64_t nb;
};

UnrolledLayout unrolled_layout(int32_t n, int32_t h, int32_t w, int64_t ld, int32_t K, int32_t c) {
    UnrolledLayout L{};
    const size_t px = (size_t)n * (size_t)h * (size_t)ld;
    L.slot = round_up(px * sizeof(float), WMC_WORKSPACE_ALIGN);
    L.ncp = K >= 1 ? (K - 1) / c : 0;
    L.nseg = c - 1 > 2 ? c - 1 : 2;
    L.nb = wmc::adjoint_blocks(h, w);
    L.off_ckpt = kStatusBytes;
    L.off_seg = L.off_ckpt + (size_t)L.ncp * L.slot;
    L.off_g = L.off_seg + (size_t)L.nseg * L.slot;
    L.off_part = L.off_g + 2 * L.slot;
    L.total = L.off_part + round_up((size_t)(K > 0 ? K : 1) * n * L.nb * sizeof(double), WMC_WORKSPACE_ALIGN);
    return L;
}

wmc_status_t check_unrolled(const float *f, const float *lambda, float step, int32_t K, int32_t c,
                            int32_t n, int32_t h, int32_t w, int64_t ld, wmc_boundary_t bnd) {
    wmc_status_t s;
    if ((s = check_enums(WMC_F32, bnd)) != WMC_OK) return s;
    if ((s = check_image(h, w, ld, "image")) != WMC_OK) return s;
    if (n < 1 || n > 65535) return fail(WMC_ERR_INVALID_ARG, "image count must be 1..65535 (got %d)", n);
    if (h < 1 || w < 1) return fail(WMC_ERR_INVALID_ARG, "empty images");
    if (K < 0) return fail(WMC_ERR_INVALID_ARG, "K must be >= 0 (got %d)", K);
    if (c < 1) return fail(WMC_ERR_INVALID_ARG, "ckpt_every must be >= 1 (got %d)", c);
    if (!std::isfinite(step) || step <= 0.0f)
        return fail(WMC_ERR_INVALID_ARG, "step must be finite and > 0 (got %g)", step);
    if (!f || !lambda) return fail(WMC_ERR_INVALID_ARG, "f or lambda is NULL");
    return WMC_OK;
}

template <typename F>
void for_each_launch(int iters, int T, F &&fn) {
    // launch k takes min(T, remaining) steps; the first reads f (role 0) as U^0, the last writes u
    // (role 1), and the ones between ping-pong between the workspace images (roles 2 and 3)
    const int nl = (iters + T - 1) / T;
    int src = 0, done = 0;
    for (int k = 0; k < nl; ++k) {
        const int s = (iters - done) < T ? (iters - done) : T;
        const int dst = (k == nl - 1) ? 1 : 2 + (k & 1);
        fn(s, src, dst);
        src = dst;
        done += s;
    }
}

}  // namespace

// ------------------------------------------------------------------ fixed device scratch
// Scratch for wmc_denoise_noalloc: one status word and one ping-pong image, in a statically
// sized device array that every GPU loading this library holds until the process exits.  Host
// code must not pass `wmc_noalloc_scratch` itself to a kernel (on the host that name is only a
// stand-in); it looks up the device address once per device below.
constexpr size_t kNoAllocScratchBytes = size_t(32) << 20;  // 32 MiB
static __device__ __align__(256) unsigned char wmc_noalloc_scratch[kNoAllocScratchBytes];

namespace {

constexpr int kMaxDevices = 64;
std::mutex g_noalloc_mutex;
void *g_noalloc_ptr[kMaxDevices] = {};

// Device address of the scratch array on the current device (resolved on the first call per
// device, with that device current).
wmc_status_t noalloc_scratch(void **out) {
    int dev = -1;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return cuda_fail(e, "cudaGetDevice");
    if (dev < 0 || dev >= kMaxDevices)
        return fail(WMC_ERR_UNSUPPORTED, "device ordinal %d beyond %d", dev, kMaxDevices);
    std::lock_guard<std::mutex> lock(g_noalloc_mutex);
    if (!g_noalloc_ptr[dev]) {
        void *ptr = nullptr;
        e = cudaGetSymbolAddress(&ptr, wmc_noalloc_scratch);
        if (e != cudaSuccess) return cuda_fail(e, "cudaGetSymbolAddress(wmc_noalloc_scratch)");
        g_noalloc_ptr[dev] = ptr;
    }
    *out = g_noalloc_ptr[dev];
    return WMC_OK;
}

}  // namespace

extern "C" {

wmc_status_t wmc_shard_lpt(const int64_t *cost, int32_t n, int32_t world, int32_t *owner,
                           int64_t *load) {
    g_last_error[0] = 0;
    if (n < 0) return fail(WMC_ERR_INVALID_ARG, "n = %d < 0", n);
    if (world < 1) return fail(WMC_ERR_INVALID_ARG, "world = %d < 1", world);
    if (n > 0 && (!cost || !owner)) return fail(WMC_ERR_INVALID_ARG, "cost or owner is NULL");
    for (int32_t i = 0; i < n; ++i)
        if (cost[i] < 0) return fail(WMC_ERR_INVALID_ARG, "cost[%d] < 0", i);
    std::vector<int32_t> order((size_t)n);
    for (int32_t i = 0; i < n; ++i) order[(size_t)i] = i;
    std::stable_sort(order.begin(), order.end(),
                     [&](int32_t a, int32_t b) { return cost[a] > cost[b]; });
    std::vector<int64_t> acc((size_t)world, 0);
    for (int32_t i : order) {
        int32_t best = 0;
        for (int32_t r = 1; r < world; ++r)
            if (acc[(size_t)r] < acc[(size_t)best]) best = r;
        owner[i] = best;
        acc[(size_t)best] += cost[i];
    }
    if (load)
        for (int32_t r = 0; r < world; ++r) load[r] = acc[(size_t)r];
    return WMC_OK;
}

const char *wmc_status_string(wmc_status_t s) {
    switch (s) {
        case WMC_OK: return "WMC_OK";
        case WMC_ERR_INVALID_ARG: return "WMC_ERR_INVALID_ARG";
        case WMC_ERR_ALIAS: return "WMC_ERR_ALIAS";
        case WMC_ERR_UNSUPPORTED: return "WMC_ERR_UNSUPPORTED";
        case WMC_ERR_CUDA: return "WMC_ERR_CUDA";
        case WMC_ERR_TIMEOUT: return "WMC_ERR_TIMEOUT";
        case WMC_ERR_WORKSPACE: return "WMC_ERR_WORKSPACE";
        default: return "WMC_ERR_UNKNOWN";
    }
}

const char *wmc_last_error(void) { return g_last_error; }

int32_t wmc_version(void) { return 100; }

static wmc_status_t eval_impl(int mode, float scale, const void *u, void *hw, int32_t h, int32_t w,
                              int64_t ld_u, int64_t ld_hw, wmc_dtype_t dtype, wmc_boundary_t bnd,
                              wmc_stream_t stream) {
    g_last_error[0] = 0;
    wmc_status_t s;
    if ((s = check_enums(dtype, bnd)) != WMC_OK) return s;
    if ((s = check_image(h, w, ld_u, "u")) != WMC_OK) return s;
    if ((s = check_image(h, w, ld_hw, "hw")) != WMC_OK) return s;
    if (h == 0 || w == 0) return WMC_OK;
    if (!u || !hw) return fail(WMC_ERR_INVALID_ARG, "NULL image pointer");
    const size_t es = elem_size(dtype);
    if (overlap(u, span_bytes(h, w, ld_u, es), hw, span_bytes(h, w, ld_hw, es)))
        return fail(WMC_ERR_ALIAS, "hw overlaps u");
    wmc::StreamParams p{};
    p.u = u;
    p.out = hw;
    p.ldu = ld_u;
    p.ldo = ld_hw;
    p.h = h;
    p.w = w;
    p.c_h = scale;
    if (mode == wmc::MODE_EVAL && dtype == WMC_F32) {
        // FP32 rows that TMA can read: the persistent kernel with double-buffered windows
        alignas(64) CUtensorMap map;
        if (encode_window_map(&map, u, dtype, h, w, ld_u)) {
            cudaError_t e = wmc::launch_eval_tma(&map, static_cast<float *>(hw), ld_hw, h, w, (int)bnd, scale,
                                                 (cudaStream_t)stream);
            if (e != cudaSuccess) return cuda_fail(e, "eval kernel launch");
            return WMC_OK;
        }
    }
    const bool vec = pair_aligned(u, ld_u, es) && pair_aligned(hw, ld_hw, es);
    cudaError_t e = wmc::launch_stream((int)dtype, mode, (int)bnd, p, vec, (cudaStream_t)stream);
    if (e != cudaSuccess) return cuda_fail(e, "eval kernel launch");
    return WMC_OK;
}

wmc_status_t wmc_eval(const void *u, void *hw, int32_t h, int32_t w, int64_t ld_u, int64_t ld_hw,
                      wmc_dtype_t dtype, wmc_boundary_t bnd, wmc_stream_t stream) {
    // the kernels carry 12 * H^w; the output scale brings it back
    return eval_impl(wmc::MODE_EVAL, 1.0f / 12.0f, u, hw, h, w, ld_u, ld_hw, dtype, bnd, stream);
}

wmc_status_t wmc_eval_status(wmc_stream_t stream) {
    g_last_error[0] = 0;
    unsigned int word = 0;
    cudaError_t e = wmc::eval_tma_status(&word, (cudaStream_t)stream);
    if (e != cudaSuccess) return cuda_fail(e, "read the evaluation status word");
    if (word & 1u) return fail(WMC_ERR_TIMEOUT, "an evaluation kernel gave up waiting for its TMA load");
    return WMC_OK;
}

wmc_status_t wmc_eval_fd(const void *u, void *hw, int32_t h, int32_t w, int64_t ld_u,
                         int64_t ld_hw, wmc_dtype_t dtype, wmc_boundary_t bnd,
                         wmc_stream_t stream) {
    return eval_impl(wmc::MODE_FD_EVAL, 1.0f, u, hw, h, w, ld_u, ld_hw, dtype, bnd, stream);
}

size_t wmc_denoise_workspace_size(int32_t h, int32_t w, int64_t ld, wmc_dtype_t dtype) {
    const size_t es = elem_size(dtype);
    if (h <= 0 || w <= 0 || ld < w || es == 0) return 0;
    // run_flow's images and status word, then the per-tile flags
    return flow_core_bytes(h, w, ld, dtype) +
           round_up((size_t)flow_flag_words(h, w) * sizeof(unsigned int), WMC_WORKSPACE_ALIGN);
}

// The flags' place in a workspace of wmc_denoise_workspace_size bytes.
unsigned int *flow_flags(void *workspace, int32_t h, int32_t w, int64_t ld, wmc_dtype_t dtype) {
    return reinterpret_cast<unsigned int *>(static_cast<char *>(workspace) + flow_core_bytes(h, w, ld, dtype));
}

wmc_status_t wmc_denoise_ex(const void *f, const void *u0, void *u, int32_t h, int32_t w,
                            int64_t ld, wmc_dtype_t dtype, float lambda, float step,
                            int32_t iters, wmc_boundary_t bnd, const wmc_config_t *config,
                            void *workspace, size_t workspace_bytes, wmc_stream_t stream) {
    g_last_error[0] = 0;
    int T = 0, tile = kDefaultTile;
    bool dflt = false;
    wmc_status_t s =
        check_flow_args(f, u0, u, h, w, ld, dtype, lambda, step, iters, bnd, config, &T, &tile, &dflt);
    if (s != WMC_OK) return s;
    if (h == 0 || w == 0) return WMC_OK;
    if (iters > 0) {
        const size_t need = wmc_denoise_workspace_size(h, w, ld, dtype);
        if (!workspace || workspace_bytes < need)
            return fail(WMC_ERR_WORKSPACE, "workspace of %zu bytes needed, %zu given", need,
                        workspace ? workspace_bytes : (size_t)0);
        if ((uintptr_t)workspace % WMC_WORKSPACE_ALIGN)
            return fail(WMC_ERR_WORKSPACE, "workspace not %d-byte aligned", WMC_WORKSPACE_ALIGN);
        const size_t n = span_bytes(h, w, ld, elem_size(dtype));
        if (overlap(workspace, need, f, n) || overlap(workspace, need, u, n) ||
            overlap(workspace, need, u0, n))
            return fail(WMC_ERR_ALIAS, "workspace overlaps an image");
    }
    return run_flow(f, u0, u, h, w, ld, dtype, lambda, step, iters, bnd, T, workspace,
                    (cudaStream_t)stream, false, tile, dflt,
                    iters > 0 ? flow_flags(workspace, h, w, ld, dtype) : nullptr);
}

int32_t wmc_denoise_cluster_size(int32_t h, int32_t w, int32_t iters) {
    g_last_error[0] = 0;
    if (iters < kClusterMinIters) return 0;
    const int ctas = wmc::cluster_ctas(h, w);
    return (ctas > 0 && wmc::cluster_fits(ctas)) ? ctas : 0;
}

wmc_status_t wmc_denoise_fd(const void *f, const void *u0, void *u, int32_t h, int32_t w, int64_t ld,
                            wmc_dtype_t dtype, float lambda, float step, int32_t iters,
                            wmc_boundary_t bnd, void *workspace, size_t workspace_bytes,
                            wmc_stream_t stream) {
    g_last_error[0] = 0;
    int T = 0;
    wmc_status_t s =
        check_flow_args(f, u0, u, h, w, ld, dtype, lambda, step, iters, bnd, nullptr, &T);
    if (s != WMC_OK) return s;
    if (h == 0 || w == 0) return WMC_OK;
    if (iters > 0) {
        const size_t need = wmc_denoise_workspace_size(h, w, ld, dtype);
        if (!workspace || workspace_bytes < need)
            return fail(WMC_ERR_WORKSPACE, "workspace of %zu bytes needed, %zu given", need,
                        workspace ? workspace_bytes : (size_t)0);
        if ((uintptr_t)workspace % WMC_WORKSPACE_ALIGN)
            return fail(WMC_ERR_WORKSPACE, "workspace not %d-byte aligned", WMC_WORKSPACE_ALIGN);
        const size_t n = span_bytes(h, w, ld, elem_size(dtype));
        if (overlap(workspace, need, f, n) || overlap(workspace, need, u, n) ||
            overlap(workspace, need, u0, n))
            return fail(WMC_ERR_ALIAS, "workspace overlaps an image");
    }
    return run_flow(f, u0, u, h, w, ld, dtype, lambda, step, iters, bnd, 1, workspace,
                    (cudaStream_t)stream, true);
}

wmc_status_t wmc_denoise(const void *f, const void *u0, void *u, int32_t h, int32_t w, int64_t ld,
                         wmc_dtype_t dtype, float lambda, float step, int32_t iters,
                         wmc_boundary_t bnd, void *workspace, size_t workspace_bytes,
                         wmc_stream_t stream) {
    return wmc_denoise_ex(f, u0, u, h, w, ld, dtype, lambda, step, iters, bnd, nullptr, workspace,
                          workspace_bytes, stream);
}

size_t wmc_denoise_host_workspace_size(int32_t h, int32_t w, int64_t ld, wmc_dtype_t dtype) {
    // f, U^0 (when given separately), U, then the ping-pong image and status word.
    if (h <= 0 || w <= 0 || ld < w || elem_size(dtype) == 0) return 0;
    return 3 * image_bytes(h, ld, dtype) + wmc_denoise_workspace_size(h, w, ld, dtype);
}

wmc_status_t wmc_denoise_host(const void *f_host, const void *u0_host, void *u_host, int32_t h,
                              int32_t w, int64_t ld, wmc_dtype_t dtype, float lambda, float step,
                              int32_t iters, wmc_boundary_t bnd, void *workspace,
                              size_t workspace_bytes, wmc_stream_t stream) {
    g_last_error[0] = 0;
    int T = 0;
    wmc_status_t s = check_flow_args(f_host, u0_host, u_host, h, w, ld, dtype, lambda, step, iters,
                                     bnd, nullptr, &T);
    if (s != WMC_OK) return s;
    if (h == 0 || w == 0) return WMC_OK;
    const size_t one = image_bytes(h, ld, dtype);
    const size_t need = wmc_denoise_host_workspace_size(h, w, ld, dtype);
    if (!workspace || workspace_bytes < need)
        return fail(WMC_ERR_WORKSPACE, "device workspace of %zu bytes needed, %zu given", need,
                    workspace ? workspace_bytes : (size_t)0);
    if ((uintptr_t)workspace % WMC_WORKSPACE_ALIGN)
        return fail(WMC_ERR_WORKSPACE, "workspace not %d-byte aligned", WMC_WORKSPACE_ALIGN);
    // [status | ping-pong image] (as wmc_denoise) followed by f, U^0 and U.
    char *base = static_cast<char *>(workspace);
    void *d_ws = base;
    base += wmc_denoise_workspace_size(h, w, ld, dtype);
    void *d_f = f_host ? base : nullptr;
    void *d_u0 = u0_host ? base + one : nullptr;
    void *d_u = base + 2 * one;
    const size_t es = elem_size(dtype);
    const size_t pitch = (size_t)ld * es;
    cudaStream_t st = (cudaStream_t)stream;
    cudaError_t e;
    if (d_f && (e = cudaMemcpy2DAsync(d_f, pitch, f_host, pitch, w * es, h, cudaMemcpyHostToDevice,
                                      st)) != cudaSuccess)
        return cuda_fail(e, "copy f to device");
    if (d_u0 && (e = cudaMemcpy2DAsync(d_u0, pitch, u0_host, pitch, w * es, h,
                                       cudaMemcpyHostToDevice, st)) != cudaSuccess)
        return cuda_fail(e, "copy u0 to device");
    s = run_flow(d_f, d_u0, d_u, h, w, ld, dtype, lambda, step, iters, bnd, T, d_ws, st, false,
                 kDefaultTile, true, flow_flags(d_ws, h, w, ld, dtype));
    if (s != WMC_OK) return s;
    if ((e = cudaMemcpy2DAsync(u_host, pitch, d_u, pitch, w * es, h, cudaMemcpyDeviceToHost, st)) !=
        cudaSuccess)
        return cuda_fail(e, "copy result to host");
    return WMC_OK;
}

wmc_status_t wmc_denoise_status(const void *workspace, wmc_stream_t stream) {
    g_last_error[0] = 0;
    if (!workspace) return fail(WMC_ERR_INVALID_ARG, "workspace is NULL");
    unsigned int word = 0;
    cudaStream_t st = (cudaStream_t)stream;
    cudaError_t e = cudaMemcpyAsync(&word, workspace, sizeof word, cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return cuda_fail(e, "read status word");
    if (word & 1u) return fail(WMC_ERR_TIMEOUT, "a tile kernel gave up waiting for its TMA load");
    return WMC_OK;
}

wmc_status_t wmc_selftest_wait_timeout(void *workspace, int64_t limit_ns, wmc_stream_t stream) {
    g_last_error[0] = 0;
    if (!workspace) return fail(WMC_ERR_INVALID_ARG, "workspace is NULL");
    if ((uintptr_t)workspace % WMC_WORKSPACE_ALIGN)
        return fail(WMC_ERR_WORKSPACE, "workspace not %d-byte aligned", WMC_WORKSPACE_ALIGN);
    if (limit_ns < 1 || limit_ns > 1000000000LL)
        return fail(WMC_ERR_INVALID_ARG, "limit_ns = %lld outside 1 .. 1e9", (long long)limit_ns);
    cudaError_t e = wmc::launch_selftest_wait(static_cast<unsigned int *>(workspace), (uint64_t)limit_ns,
                                              (cudaStream_t)stream);
    if (e != cudaSuccess) return cuda_fail(e, "self-test wait kernel launch");
    return WMC_OK;
}

size_t wmc_energy_workspace_size(int32_t h, int32_t w) {
    if (h <= 0 || w <= 0) return WMC_WORKSPACE_ALIGN;
    return WMC_WORKSPACE_ALIGN +
           round_up(3 * sizeof(double) * (size_t)wmc::energy_blocks(h, w), WMC_WORKSPACE_ALIGN);
}

wmc_status_t wmc_energy(const void *u, const void *f, const void *clean, int32_t h, int32_t w,
                        int64_t ld, wmc_dtype_t dtype, wmc_boundary_t bnd, double *out,
                        void *workspace, size_t workspace_bytes, wmc_stream_t stream) {
    g_last_error[0] = 0;
    wmc_status_t s;
    if ((s = check_enums(dtype, bnd)) != WMC_OK) return s;
    if ((s = check_image(h, w, ld, "u")) != WMC_OK) return s;
    if (!out) return fail(WMC_ERR_INVALID_ARG, "out is NULL");
    cudaStream_t st = (cudaStream_t)stream;
    if (h == 0 || w == 0) {
        cudaError_t e = cudaMemsetAsync(out, 0, 3 * sizeof(double), st);
        return e == cudaSuccess ? WMC_OK : cuda_fail(e, "clear out");
    }
    if (!u) return fail(WMC_ERR_INVALID_ARG, "u is NULL");
    const size_t need = wmc_energy_workspace_size(h, w);
    if (!workspace || workspace_bytes < need)
        return fail(WMC_ERR_WORKSPACE, "workspace of %zu bytes needed", need);
    if ((uintptr_t)workspace % WMC_WORKSPACE_ALIGN)
        return fail(WMC_ERR_WORKSPACE, "workspace not %d-byte aligned", WMC_WORKSPACE_ALIGN);
#ifndef WMC_ENERGY_TMA
#define WMC_ENERGY_TMA 1  // 0: FP32 energies take the streaming kernels only
#endif
    if (WMC_ENERGY_TMA && dtype == WMC_F32) {
        // FP32 rows that TMA can read: the persistent kernel fed by TMA windows (U) and boxes
        // (f, clean)
        alignas(64) CUtensorMap maps[3];
        memset(maps, 0, sizeof maps);
        int bw = 0, bh = 0;
        wmc::energy_tma_box(&bw, &bh);
        const bool ok = encode_window_map(&maps[0], u, dtype, h, w, ld) &&
                        (!f || encode_box_map(&maps[1], f, dtype, h, w, ld, bw, bh)) &&
                        (!clean || encode_box_map(&maps[2], clean, dtype, h, w, ld, bw, bh));
        if (ok) {
            cudaError_t e = wmc::launch_energy_tma(maps, f != nullptr, clean != nullptr, h, w, (int)bnd, out,
                                                   workspace, st);
            if (e != cudaSuccess) return cuda_fail(e, "energy kernel launch");
            return WMC_OK;
        }
    }
    cudaError_t e = wmc::launch_energy((int)dtype, u, f, clean, h, w, ld, (int)bnd, out, workspace, st);
    if (e != cudaSuccess) return cuda_fail(e, "energy kernel launch");
    return WMC_OK;
}

size_t wmc_batch_workspace_size(const wmc_image_t *imgs, int32_t n, wmc_dtype_t dtype,
                                const wmc_config_t *config) {
    if (n < 0 || (n > 0 && !imgs) || elem_size(dtype) == 0) return 0;
    const int T = batch_steps(config);
    if (T < 1 || T > wmc::kMaxSteps) return 0;
    for (int32_t i = 0; i < n; ++i)
        if (imgs[i].h < 0 || imgs[i].w < 0 || (imgs[i].h > 0 && imgs[i].w > 0 && imgs[i].ld < imgs[i].w))
            return 0;
    const int tile = batch_tile(config);
    if (tile < 1 || tile > kTileShapes) return 0;
    return batch_layout(imgs, n, dtype, T, tile).total;
}

wmc_status_t wmc_batch_plan(const wmc_image_t *imgs, int32_t n, wmc_dtype_t dtype,
                            wmc_boundary_t bnd, const wmc_config_t *config, void *workspace,
                            size_t workspace_bytes, wmc_batch_t *plan, wmc_stream_t stream) {
    g_last_error[0] = 0;
    if (!plan) return fail(WMC_ERR_INVALID_ARG, "plan is NULL");
    memset(plan, 0, sizeof *plan);
    wmc_status_t s = check_batch(imgs, n, dtype, bnd, config);
    if (s != WMC_OK) return s;
    const int T = batch_steps(config);
    const int tile = batch_tile(config);
    const BatchLayout L = batch_layout(imgs, n, dtype, T, tile);
    if (!workspace || workspace_bytes < L.total)
        return fail(WMC_ERR_WORKSPACE, "workspace of %zu bytes needed, %zu given", L.total,
                    workspace ? workspace_bytes : (size_t)0);
    if ((uintptr_t)workspace % WMC_WORKSPACE_ALIGN)
        return fail(WMC_ERR_WORKSPACE, "workspace not %d-byte aligned", WMC_WORKSPACE_ALIGN);
    const size_t es = elem_size(dtype);
    for (int32_t i = 0; i < n; ++i) {
        if (imgs[i].h == 0 || imgs[i].w == 0) continue;
        const size_t nb = span_bytes(imgs[i].h, imgs[i].w, imgs[i].ld, es);
        if (overlap(workspace, L.total, imgs[i].f, nb) || overlap(workspace, L.total, imgs[i].u, nb))
            return fail(WMC_ERR_ALIAS, "workspace overlaps image %d", i);
    }
    int owt, oht;
    out_tile(T, tile, &owt, &oht);
    char *base = static_cast<char *>(workspace);
    std::vector<wmc::BatchImage> desc((size_t)n);
    bool any_copy = false;
    std::vector<int4> tiles;
    tiles.reserve((size_t)L.ntiles);
    for (int32_t i = 0; i < n; ++i) {
        const wmc_image_t &m = imgs[i];
        wmc::BatchImage &d = desc[i];
        memset(&d, 0, sizeof d);
        if (m.h == 0 || m.w == 0) continue;
        const size_t one = image_bytes(m.h, L.ld_read[i], dtype);
        d.copy_f = L.copy_f[i];
        d.f_src = m.f;
        d.buf[0] = d.copy_f ? base + L.buf_off[i] + 2 * one : m.f;
        d.buf[1] = m.u;
        d.buf[2] = base + L.buf_off[i];
        d.buf[3] = base + L.buf_off[i] + one;
        d.ld = L.ld_read[i];
        d.ld_out = m.ld;
        d.h = m.h;
        d.w = m.w;
        d.c_keep = 1.0f - m.step;
        d.c_f = m.step;
        d.c_h = m.step * m.lambda / 12.0f;
        for (int r = 0; r < 4; ++r)
            d.use_tma[r] = r != 1 && encode_window_map(&d.map[r], d.buf[r], dtype, m.h, m.w, d.ld, tile) ? 1 : 0;
        any_copy |= d.copy_f != 0;
        for (int y0 = 0; y0 < m.h; y0 += oht)
            for (int x0 = 0; x0 < m.w; x0 += owt) tiles.push_back(make_int4(i, x0, y0, 0));
    }
    cudaStream_t st = (cudaStream_t)stream;
    cudaError_t e = cudaSuccess;
    if (n > 0)
        e = cudaMemcpyAsync(base + L.off_images, desc.data(), desc.size() * sizeof(wmc::BatchImage),
                            cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess && !tiles.empty())
        e = cudaMemcpyAsync(base + L.off_tiles, tiles.data(), tiles.size() * sizeof(int4),
                            cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return cuda_fail(e, "upload batch plan");
    BatchPlan bp{};
    bp.ws = workspace;
    bp.ntiles = L.ntiles;
    bp.off_images = (int64_t)L.off_images;
    bp.off_tiles = (int64_t)L.off_tiles;
    bp.n = n;
    bp.dtype = (int32_t)dtype;
    bp.bnd = (int32_t)bnd;
    bp.steps = T;
    bp.owt = owt;
    bp.oht = oht;
    bp.tile = tile;
    bp.any_copy = any_copy ? 1 : 0;
    bp.magic = kBatchMagic;
    memcpy(plan, &bp, sizeof bp);
    return WMC_OK;
}

wmc_status_t wmc_batch_run(const wmc_batch_t *plan, int32_t iters, wmc_stream_t stream) {
    g_last_error[0] = 0;
    if (!plan) return fail(WMC_ERR_INVALID_ARG, "plan is NULL");
    BatchPlan bp;
    memcpy(&bp, plan, sizeof bp);
    if (bp.magic != kBatchMagic) return fail(WMC_ERR_INVALID_ARG, "plan was not made by wmc_batch_plan");
    if (iters < 0) return fail(WMC_ERR_INVALID_ARG, "iters must be >= 0 (got %d)", iters);
    if (bp.ntiles == 0) return WMC_OK;
    cudaStream_t st = (cudaStream_t)stream;
    char *base = static_cast<char *>(bp.ws);
    unsigned int *status = reinterpret_cast<unsigned int *>(base);
    cudaError_t e = cudaMemsetAsync(status, 0, sizeof(unsigned int), st);
    if (e != cudaSuccess) return cuda_fail(e, "clear status");
    wmc::TileParams p{};
    p.images = reinterpret_cast<const wmc::BatchImage *>(base + bp.off_images);
    p.tiles = reinterpret_cast<const int4 *>(base + bp.off_tiles);
    p.owt = bp.owt;
    p.oht = bp.oht;
    p.status = status;
    if (bp.ntiles > 0x7fffffffLL) return fail(WMC_ERR_INVALID_ARG, "too many tiles");
    const int es = (int)elem_size((wmc_dtype_t)bp.dtype);
    auto copy = [&](int to_u) {
        if (es == 4)
            batch_copy_kernel<uint32_t><<<(unsigned)bp.ntiles, 256, 0, st>>>(p.images, p.tiles, bp.owt, bp.oht, to_u);
        else
            batch_copy_kernel<uint16_t><<<(unsigned)bp.ntiles, 256, 0, st>>>(p.images, p.tiles, bp.owt, bp.oht, to_u);
        return cudaGetLastError();
    };
    if (iters == 0) {  // U^0 = f: copy every output tile
        e = copy(1);
        return e == cudaSuccess ? WMC_OK : cuda_fail(e, "batch copy launch");
    }
    // the images whose f the kernels cannot read through TMA read the workspace copy, taken now
    // (f may have changed since the plan or the last run)
    if (bp.any_copy && (e = copy(0)) != cudaSuccess) return cuda_fail(e, "batch copy launch");
    int launches = 0;
    for_each_launch(iters, bp.steps, [&](int s, int src, int dst) {
        if (e != cudaSuccess) return;
        p.src_role = src;
        p.dst_role = dst;
        p.pdl = launches++ > 0 ? 1 : 0;  // follows a tile launch: may overlap its tail
        e = launch_tile((wmc_dtype_t)bp.dtype, (wmc_boundary_t)bp.bnd, bp.tile, s, nullptr, p, bp.ntiles, st);
    });
    if (e != cudaSuccess) return cuda_fail(e, "batch kernel launch");
    return WMC_OK;
}

wmc_status_t wmc_denoise_batched(const wmc_image_t *imgs, int32_t n, wmc_dtype_t dtype,
                                 int32_t iters, wmc_boundary_t bnd, void *workspace,
                                 size_t workspace_bytes, wmc_stream_t stream) {
    wmc_batch_t plan;
    wmc_status_t s =
        wmc_batch_plan(imgs, n, dtype, bnd, nullptr, workspace, workspace_bytes, &plan, stream);
    if (s != WMC_OK) return s;
    return wmc_batch_run(&plan, iters, stream);
}

size_t wmc_batch_autotune_workspace_size(const wmc_image_t *imgs, int32_t n, wmc_dtype_t dtype) {
    size_t best = 0;
    for (int tile = 1; tile <= kTileShapes; ++tile)
        for (int T = 1; T <= wmc::kMaxSteps; ++T) {
            wmc_config_t c{T, tile};
            const size_t b = wmc_batch_workspace_size(imgs, n, dtype, &c);
            if (b == 0) return 0;
            best = b > best ? b : best;
        }
    return best;
}

// Times each candidate configuration on the caller's batch and keeps the fastest per iteration.
static wmc_status_t autotune_configs(const wmc_image_t *imgs, int32_t n, wmc_dtype_t dtype,
                                     wmc_boundary_t bnd, const wmc_config_t *cands, int32_t nc,
                                     int32_t trial_iters, void *workspace, size_t workspace_bytes,
                                     wmc_config_t *best, float *ms_per_iter, wmc_stream_t stream) {
    if (trial_iters < 1) return fail(WMC_ERR_INVALID_ARG, "trial_iters must be >= 1 (got %d)", trial_iters);
    cudaStream_t st = (cudaStream_t)stream;
    cudaEvent_t a = nullptr, b = nullptr;
    cudaError_t e = cudaEventCreate(&a);
    if (e == cudaSuccess) e = cudaEventCreate(&b);
    if (e != cudaSuccess) {
        if (a) cudaEventDestroy(a);
        return cuda_fail(e, "event create");
    }
    float best_ms = 0.0f;
    int best_k = -1;
    wmc_status_t s = WMC_OK;
    for (int32_t k = 0; k < nc && s == WMC_OK; ++k) {
        const wmc_config_t c = cands[k];
        const int T = batch_steps(&c);
        wmc_batch_t plan;
        s = wmc_batch_plan(imgs, n, dtype, bnd, &c, workspace, workspace_bytes, &plan, stream);
        if (s != WMC_OK) break;
        // one untimed run (first-launch costs), then the timed one; each covers whole launches
        const int it = ((trial_iters + T - 1) / T) * T;
        if ((s = wmc_batch_run(&plan, T, stream)) != WMC_OK) break;
        if ((e = cudaEventRecord(a, st)) != cudaSuccess) { s = cuda_fail(e, "event record"); break; }
        if ((s = wmc_batch_run(&plan, it, stream)) != WMC_OK) break;
        if ((e = cudaEventRecord(b, st)) != cudaSuccess || (e = cudaEventSynchronize(b)) != cudaSuccess) {
            s = cuda_fail(e, "event sync");
            break;
        }
        float ms = 0.0f;
        if ((e = cudaEventElapsedTime(&ms, a, b)) != cudaSuccess) { s = cuda_fail(e, "event time"); break; }
        const float per_iter = ms / (float)it;
        if (ms_per_iter) ms_per_iter[k] = per_iter;
        if (best_k < 0 || per_iter < best_ms) {
            best_ms = per_iter;
            best_k = k;
        }
        const unsigned int *status = static_cast<const unsigned int *>(workspace);
        unsigned int hs = 0;
        if ((e = cudaMemcpy(&hs, status, sizeof hs, cudaMemcpyDeviceToHost)) != cudaSuccess) {
            s = cuda_fail(e, "read status");
            break;
        }
        if (hs) s = fail(WMC_ERR_TIMEOUT, "a tile load timed out during the trial of tile %d, %d steps per launch",
                         c.tile, T);
    }
    cudaEventDestroy(a);
    cudaEventDestroy(b);
    if (s != WMC_OK) return s;
    *best = cands[best_k];
    return WMC_OK;
}

wmc_status_t wmc_batch_autotune(const wmc_image_t *imgs, int32_t n, wmc_dtype_t dtype,
                                wmc_boundary_t bnd, const int32_t *candidates, int32_t n_candidates,
                                int32_t trial_iters, void *workspace, size_t workspace_bytes,
                                wmc_config_t *best, float *ms_per_iter, wmc_stream_t stream) {
    g_last_error[0] = 0;
    static const int32_t kDefaultCandidates[] = {2, 3, 4, 5, 6, 8};
    if (!best) return fail(WMC_ERR_INVALID_ARG, "best is NULL");
    if (!candidates) {
        candidates = kDefaultCandidates;
        n_candidates = (int32_t)(sizeof kDefaultCandidates / sizeof kDefaultCandidates[0]);
    }
    if (n_candidates < 1 || n_candidates > 64)
        return fail(WMC_ERR_INVALID_ARG, "n_candidates must be 1..64 (got %d)", n_candidates);
    wmc_config_t cands[64];
    for (int32_t k = 0; k < n_candidates; ++k) {
        if (candidates[k] < 1 || candidates[k] > wmc::kMaxSteps)
            return fail(WMC_ERR_INVALID_ARG, "candidate %d: steps per launch must be 1..%d (got %d)", k,
                        wmc::kMaxSteps, candidates[k]);
        cands[k] = wmc_config_t{candidates[k], 0};
    }
    return autotune_configs(imgs, n, dtype, bnd, cands, n_candidates, trial_iters, workspace,
                            workspace_bytes, best, ms_per_iter, stream);
}

wmc_status_t wmc_batch_autotune_configs(const wmc_image_t *imgs, int32_t n, wmc_dtype_t dtype,
                                        wmc_boundary_t bnd, const wmc_config_t *candidates,
                                        int32_t n_candidates, int32_t trial_iters, void *workspace,
                                        size_t workspace_bytes, wmc_config_t *best, float *ms_per_iter,
                                        wmc_stream_t stream) {
    g_last_error[0] = 0;
    if (!best) return fail(WMC_ERR_INVALID_ARG, "best is NULL");
    wmc_config_t cands[64];
    if (!candidates) {
        static const int32_t kSteps[] = {2, 3, 4, 5, 6, 8};
        n_candidates = 0;
        for (int tile = 1; tile <= kTileShapes; ++tile)
            for (int32_t T : kSteps) cands[n_candidates++] = wmc_config_t{T, tile};
    } else {
        if (n_candidates < 1 || n_candidates > 64)
            return fail(WMC_ERR_INVALID_ARG, "n_candidates must be 1..64 (got %d)", n_candidates);
        for (int32_t k = 0; k < n_candidates; ++k) {
            const wmc_config_t &c = candidates[k];
            if (c.steps_per_launch < 1 || c.steps_per_launch > wmc::kMaxSteps || c.tile < 0 ||
                c.tile > kTileShapes)
                return fail(WMC_ERR_INVALID_ARG, "candidate %d: {steps %d, tile %d} outside {1..%d, 0..%d}", k,
                            c.steps_per_launch, c.tile, wmc::kMaxSteps, kTileShapes);
            cands[k] = c;
        }
    }
    return autotune_configs(imgs, n, dtype, bnd, cands, n_candidates, trial_iters, workspace,
                            workspace_bytes, best, ms_per_iter, stream);
}

size_t wmc_denoise_l1_workspace_size(int32_t h, int32_t w, int64_t ld) {
    if (h < 0 || w < 0 || ld < w) return 0;
    return kStatusBytes + 2 * image_bytes(h, ld, WMC_F32);
}

wmc_status_t wmc_denoise_l1(const float *f, const float *u0, float *u, float *d, int32_t h, int32_t w,
                            int64_t ld, float lambda, float step, float alpha, int32_t iters,
                            wmc_boundary_t bnd, void *workspace, size_t workspace_bytes,
                            wmc_stream_t stream) {
    g_last_error[0] = 0;
    wmc_status_t s;
    if ((s = check_enums(WMC_F32, bnd)) != WMC_OK) return s;
    if ((s = check_image(h, w, ld, "image")) != WMC_OK) return s;
    if (!std::isfinite(lambda) || lambda < 0.0f)
        return fail(WMC_ERR_INVALID_ARG, "lambda must be finite and >= 0 (got %g)", lambda);
    if (!std::isfinite(step) || step <= 0.0f)
        return fail(WMC_ERR_INVALID_ARG, "step must be finite and > 0 (got %g)", step);
    if (!std::isfinite(alpha) || alpha <= 0.0f)
        return fail(WMC_ERR_INVALID_ARG, "alpha must be finite and > 0 (got %g)", alpha);
    if (iters < 0) return fail(WMC_ERR_INVALID_ARG, "iters must be >= 0 (got %d)", iters);
    if (h == 0 || w == 0) return WMC_OK;
    if (!f || !u) return fail(WMC_ERR_INVALID_ARG, "f or u is NULL");
    if (!u0) u0 = f;
    const size_t n = span_bytes(h, w, ld, 4);
    if (overlap(u, n, f, n)) return fail(WMC_ERR_ALIAS, "u overlaps f");
    if (u0 != u && overlap(u, n, u0, n)) return fail(WMC_ERR_ALIAS, "u overlaps u0");
    if (d && (overlap(d, n, f, n) || overlap(d, n, u, n) || overlap(d, n, u0, n)))
        return fail(WMC_ERR_ALIAS, "d overlaps f, u or u0");
    const size_t need = wmc_denoise_l1_workspace_size(h, w, ld);
    if (!workspace || workspace_bytes < need)
        return fail(WMC_ERR_WORKSPACE, "workspace of %zu bytes needed", need);
    if ((uintptr_t)workspace % WMC_WORKSPACE_ALIGN)
        return fail(WMC_ERR_WORKSPACE, "workspace not %d-byte aligned", WMC_WORKSPACE_ALIGN);
    if (overlap(workspace, need, f, n) || overlap(workspace, need, u, n) ||
        overlap(workspace, need, u0, n) || (d && overlap(workspace, need, d, n)))
        return fail(WMC_ERR_ALIAS, "workspace overlaps an image");
    cudaStream_t st = (cudaStream_t)stream;
    char *base = static_cast<char *>(workspace) + kStatusBytes;
    float *tmp = reinterpret_cast<float *>(base);
    float *dw = d ? d : reinterpret_cast<float *>(base + image_bytes(h, ld, WMC_F32));
    cudaError_t e;
    if (!d) {  // d^0 = 0
        e = cudaMemset2DAsync(dw, ld * 4, 0, w * 4, h, st);
        if (e != cudaSuccess) return cuda_fail(e, "clear d");
    }
    const float *src = u0;
    if (iters == 0) {
        if (u0 != u) {
            e = cudaMemcpy2DAsync(u, ld * 4, u0, ld * 4, w * 4, h, cudaMemcpyDeviceToDevice, st);
            if (e != cudaSuccess) return cuda_fail(e, "copy U^0");
        }
        return WMC_OK;
    }
    // step t writes u when iters-1-t is even, so the last step lands in u; U^0 read from u itself
    // is moved to the workspace first when the first step would overwrite it
    if (u0 == u && ((iters - 1) % 2 == 0)) {
        e = cudaMemcpy2DAsync(tmp, ld * 4, u, ld * 4, w * 4, h, cudaMemcpyDeviceToDevice, st);
        if (e != cudaSuccess) return cuda_fail(e, "copy U^0");
        src = tmp;
    }
    const bool vec = pair_aligned(src, ld, 4) && pair_aligned(f, ld, 4) && pair_aligned(u, ld, 4) &&
                     pair_aligned(tmp, ld, 4) && pair_aligned(dw, ld, 4);
    const float c_h = step * lambda / 12.0f, c_d = step / alpha;
    for (int32_t t = 0; t < iters; ++t) {
        float *dst = ((iters - 1 - t) % 2 == 0) ? u : tmp;
        e = wmc::launch_l1_step((int)bnd, src, f, dw, dst, h, w, ld, c_h, c_d, alpha, vec, st);
        if (e != cudaSuccess) return cuda_fail(e, "primal-dual step");
        src = dst;
    }
    return WMC_OK;
}

size_t wmc_unrolled_workspace_size(int32_t n, int32_t h, int32_t w, int64_t ld, int32_t K,
                                   int32_t ckpt_every) {
    if (n < 1 || h < 1 || w < 1 || ld < w || K < 0 || ckpt_every < 1) return 0;
    return unrolled_layout(n, h, w, ld, K, ckpt_every).total;
}

wmc_status_t wmc_unrolled_forward(const float *f, const float *lambda, float step, int32_t K,
                                  int32_t ckpt_every, int32_t n, int32_t h, int32_t w, int64_t ld,
                                  wmc_boundary_t bnd, float *u, void *workspace,
                                  size_t workspace_bytes, wmc_stream_t stream) {
    g_last_error[0] = 0;
    wmc_status_t s = check_unrolled(f, lambda, step, K, ckpt_every, n, h, w, ld, bnd);
    if (s != WMC_OK) return s;
    if (!u) return fail(WMC_ERR_INVALID_ARG, "u is NULL");
    const int64_t stride = (int64_t)h * ld;
    const size_t nbytes = span_bytes(n * h, w, ld, 4);
    if (overlap(u, nbytes, f, nbytes)) return fail(WMC_ERR_ALIAS, "u overlaps f");
    const UnrolledLayout L = unrolled_layout(n, h, w, ld, K, ckpt_every);
    if (!workspace || workspace_bytes < L.total)
        return fail(WMC_ERR_WORKSPACE, "workspace of %zu bytes needed", L.total);
    if ((uintptr_t)workspace % WMC_WORKSPACE_ALIGN)
        return fail(WMC_ERR_WORKSPACE, "workspace not %d-byte aligned", WMC_WORKSPACE_ALIGN);
    if (overlap(workspace, L.total, f, nbytes) || overlap(workspace, L.total, u, nbytes))
        return fail(WMC_ERR_ALIAS, "workspace overlaps an image");
    cudaStream_t st = (cudaStream_t)stream;
    char *base = static_cast<char *>(workspace);
    cudaError_t e;
    if (K == 0) {
        e = cudaMemcpy2DAsync(u, ld * 4, f, ld * 4, w * 4, (size_t)n * h, cudaMemcpyDeviceToDevice, st);
        return e == cudaSuccess ? WMC_OK : cuda_fail(e, "copy U^0");
    }
    const bool vec = pair_aligned(f, ld, 4) && pair_aligned(u, ld, 4);
    float *tmp[2] = {reinterpret_cast<float *>(base + L.off_seg),
                     reinterpret_cast<float *>(base + L.off_seg + L.slot)};
    const float *src = f;
    for (int32_t t = 0; t < K; ++t) {
        float *dst;
        if (t + 1 == K)
            dst = u;
        else if ((t + 1) % ckpt_every == 0)
            dst = reinterpret_cast<float *>(base + L.off_ckpt + (size_t)((t + 1) / ckpt_every - 1) * L.slot);
        else
            dst = (src == tmp[0]) ? tmp[1] : tmp[0];
        e = wmc::launch_stack_step((int)bnd, src, f, dst, lambda, step, n, h, w, ld, stride, vec, st);
        if (e != cudaSuccess) return cuda_fail(e, "unrolled forward step");
        src = dst;
    }
    return WMC_OK;
}

wmc_status_t wmc_unrolled_backward(const float *f, const float *lambda, float step, int32_t K,
                                   int32_t ckpt_every, int32_t n, int32_t h, int32_t w, int64_t ld,
                                   wmc_boundary_t bnd, const float *grad_u, float *grad_f,
                                   float *grad_lambda, void *workspace, size_t workspace_bytes,
                                   wmc_stream_t stream) {
    g_last_error[0] = 0;
    wmc_status_t s = check_unrolled(f, lambda, step, K, ckpt_every, n, h, w, ld, bnd);
    if (s != WMC_OK) return s;
    if (!grad_u || !grad_f || !grad_lambda)
        return fail(WMC_ERR_INVALID_ARG, "grad_u, grad_f or grad_lambda is NULL");
    const int64_t stride = (int64_t)h * ld;
    const size_t nbytes = span_bytes(n * h, w, ld, 4);
    if (overlap(grad_f, nbytes, grad_u, nbytes) || overlap(grad_f, nbytes, f, nbytes))
        return fail(WMC_ERR_ALIAS, "grad_f overlaps grad_u or f");
    const UnrolledLayout L = unrolled_layout(n, h, w, ld, K, ckpt_every);
    if (!workspace || workspace_bytes < L.total)
        return fail(WMC_ERR_WORKSPACE, "workspace of %zu bytes needed", L.total);
    if ((uintptr_t)workspace % WMC_WORKSPACE_ALIGN)
        return fail(WMC_ERR_WORKSPACE, "workspace not %d-byte aligned", WMC_WORKSPACE_ALIGN);
    if (overlap(workspace, L.total, f, nbytes) || overlap(workspace, L.total, grad_u, nbytes) ||
        overlap(workspace, L.total, grad_f, nbytes))
        return fail(WMC_ERR_ALIAS, "workspace overlaps f, grad_u or grad_f");
    cudaStream_t st = (cudaStream_t)stream;
    cudaError_t e;
    if (K == 0) {
        e = cudaMemcpy2DAsync(grad_f, ld * 4, grad_u, ld * 4, w * 4, (size_t)n * h,
                              cudaMemcpyDeviceToDevice, st);
        if (e == cudaSuccess) e = cudaMemsetAsync(grad_lambda, 0, (size_t)n * sizeof(float), st);
        return e == cudaSuccess ? WMC_OK : cuda_fail(e, "K = 0 backward");
    }
    char *base = static_cast<char *>(workspace);
    const bool vec = pair_aligned(f, ld, 4);
    auto ckpt = [&](int i) { return reinterpret_cast<float *>(base + L.off_ckpt + (size_t)i * L.slot); };
    auto seg = [&](int i) { return reinterpret_cast<float *>(base + L.off_seg + (size_t)i * L.slot); };
    float *gbuf[2] = {reinterpret_cast<float *>(base + L.off_g),
                      reinterpret_cast<float *>(base + L.off_g + L.slot)};
    double *part = reinterpret_cast<double *>(base + L.off_part);
    const float *g_in = grad_u;
    int gi = 0;
    const int c = ckpt_every;
    const int nsegs = (K + c - 1) / c;
    for (int sgi = nsegs - 1; sgi >= 0; --sgi) {
        const int t0 = sgi * c, t1 = (t0 + c < K) ? t0 + c : K;
        const float *start = (sgi == 0) ? f : ckpt(sgi - 1);
        // recompute U^{t0+1} .. U^{t1-1} of this segment
        const float *prev = start;
        for (int j = 1; j < t1 - t0; ++j) {
            e = wmc::launch_stack_step((int)bnd, prev, f, seg(j - 1), lambda, step, n, h, w, ld, stride,
                                       vec, st);
            if (e != cudaSuccess) return cuda_fail(e, "recompute step");
            prev = seg(j - 1);
        }
        for (int t = t1 - 1; t >= t0; --t) {
            const float *Ut = (t == t0) ? start : seg(t - t0 - 1);
            float *g_out = gbuf[gi];
            e = wmc::launch_adjoint_step((int)bnd, Ut, g_in, g_out, grad_f, part + (size_t)t * n * L.nb,
                                         lambda, step, t == K - 1, t == 0, n, h, w, ld, stride, st);
            if (e != cudaSuccess) return cuda_fail(e, "adjoint step");
            g_in = g_out;
            gi ^= 1;
        }
    }
    e = wmc::launch_lambda_grad(part, K, n, L.nb, step, grad_lambda, st);
    if (e != cudaSuccess) return cuda_fail(e, "dlambda reduction");
    return WMC_OK;
}

wmc_status_t wmc_energy_grad(const float *u, float *grad, int32_t h, int32_t w, int64_t ld,
                             wmc_boundary_t bnd, wmc_stream_t stream) {
    g_last_error[0] = 0;
    wmc_status_t s;
    if ((s = check_enums(WMC_F32, bnd)) != WMC_OK) return s;
    if ((s = check_image(h, w, ld, "u")) != WMC_OK) return s;
    if (h == 0 || w == 0) return WMC_OK;
    if (!u || !grad) return fail(WMC_ERR_INVALID_ARG, "NULL image pointer");
    const size_t nbytes = span_bytes(h, w, ld, 4);
    if (overlap(u, nbytes, grad, nbytes)) return fail(WMC_ERR_ALIAS, "grad overlaps u");
    cudaError_t e = wmc::launch_energy_grad((int)bnd, u, grad, h, w, ld, (cudaStream_t)stream);
    return e == cudaSuccess ? WMC_OK : cuda_fail(e, "energy gradient");
}

size_t wmc_denoise_noalloc_max_bytes(void) { return kNoAllocScratchBytes; }

wmc_status_t wmc_denoise_noalloc(const void *f, const void *u0, void *u, int32_t h, int32_t w,
                                 int64_t ld, wmc_dtype_t dtype, float lambda, float step,
                                 int32_t iters, wmc_boundary_t bnd, wmc_stream_t stream) {
    g_last_error[0] = 0;
    int T = 0;
    wmc_status_t s =
        check_flow_args(f, u0, u, h, w, ld, dtype, lambda, step, iters, bnd, nullptr, &T);
    if (s != WMC_OK) return s;
    if (h == 0 || w == 0) return WMC_OK;
    // (this entry point chains its launches without the per-tile flags, which the size counts)
    const size_t need = wmc_denoise_workspace_size(h, w, ld, dtype);
    if (need > kNoAllocScratchBytes)
        return fail(WMC_ERR_INVALID_ARG,
                    "image needs %zu bytes of scratch; the fixed device scratch of "
                    "wmc_denoise_noalloc holds %zu bytes (use wmc_denoise with a workspace)",
                    need, kNoAllocScratchBytes);
    void *scratch = nullptr;
    if ((s = noalloc_scratch(&scratch)) != WMC_OK) return s;
    // run_flow clears the status word at the start of every call; nothing else in the scratch
    // needs a defined value (the ping-pong image is always written before it is read)
    return run_flow(f, u0, u, h, w, ld, dtype, lambda, step, iters, bnd, T, scratch,
                    (cudaStream_t)stream, false, kDefaultTile, true);
}

wmc_status_t wmc_denoise_noalloc_status(wmc_stream_t stream) {
    g_last_error[0] = 0;
    void *scratch = nullptr;
    wmc_status_t s = noalloc_scratch(&scratch);
    if (s != WMC_OK) return s;
    return wmc_denoise_status(scratch, stream);
}

wmc_status_t wmc_selftest_status_timeout(int32_t target, int64_t limit_ns, wmc_stream_t stream) {
    g_last_error[0] = 0;
    if (limit_ns < 1 || limit_ns > 1000000000LL)
        return fail(WMC_ERR_INVALID_ARG, "limit_ns = %lld outside 1 .. 1e9", (long long)limit_ns);
    unsigned int *word = nullptr;
    if (target == WMC_SELFTEST_EVAL) {
        cudaError_t e = wmc::eval_status_word(&word);
        if (e != cudaSuccess) return cuda_fail(e, "evaluation status word");
    } else if (target == WMC_SELFTEST_NOALLOC) {
        void *scratch = nullptr;
        wmc_status_t s = noalloc_scratch(&scratch);
        if (s != WMC_OK) return s;
        word = static_cast<unsigned int *>(scratch);
    } else {
        return fail(WMC_ERR_INVALID_ARG, "unknown self-test target %d", target);
    }
    cudaError_t e = wmc::launch_selftest_wait(word, (uint64_t)limit_ns, (cudaStream_t)stream);
    if (e != cudaSuccess) return cuda_fail(e, "self-test wait kernel launch");
    return WMC_OK;
}

wmc_status_t wmc_selftest_flag_timeout(const void *f, void *u, int32_t h, int32_t w, int64_t ld,
                                       void *workspace, size_t workspace_bytes, wmc_stream_t stream) {
    g_last_error[0] = 0;
    int T = 0;
    wmc_status_t s = check_flow_args(f, nullptr, u, h, w, ld, WMC_F32, 1.0f, 0.25f, 4,
                                     WMC_BOUNDARY_REPLICATE, nullptr, &T);
    if (s != WMC_OK) return s;
    if (h == 0 || w == 0) return fail(WMC_ERR_INVALID_ARG, "empty image");
    if (!f) return fail(WMC_ERR_INVALID_ARG, "f is NULL");
    const size_t need = wmc_denoise_workspace_size(h, w, ld, WMC_F32);
    if (!workspace || workspace_bytes < need)
        return fail(WMC_ERR_WORKSPACE, "workspace of %zu bytes needed, %zu given", need,
                    workspace ? workspace_bytes : (size_t)0);
    if ((uintptr_t)workspace % WMC_WORKSPACE_ALIGN)
        return fail(WMC_ERR_WORKSPACE, "workspace not %d-byte aligned", WMC_WORKSPACE_ALIGN);
    const size_t n = span_bytes(h, w, ld, sizeof(float));
    if (overlap(workspace, need, f, n) || overlap(workspace, need, u, n))
        return fail(WMC_ERR_ALIAS, "workspace overlaps an image");
    alignas(64) CUtensorMap maps[2];
    memset(maps, 0, sizeof maps);
    if (!encode_window_map(&maps[0], f, WMC_F32, h, w, ld) || !encode_window_map(&maps[1], f, WMC_F32, h, w, ld))
        return fail(WMC_ERR_UNSUPPORTED, "f must be readable by TMA (16-byte aligned start and pitch)");
    cudaStream_t st = (cudaStream_t)stream;
    unsigned int *status = static_cast<unsigned int *>(workspace);
    unsigned int *flags = flow_flags(workspace, h, w, ld, WMC_F32);
    cudaError_t e = cudaMemsetAsync(status, 0, sizeof(unsigned int), st);
    if (e == cudaSuccess)
        e = cudaMemsetAsync(flags, 0, (size_t)flow_flag_words(h, w) * sizeof(unsigned int), st);
    if (e != cudaSuccess) return cuda_fail(e, "clear status word and tile flags");
    // the coefficients of wmc_denoise with lambda 1, step 0.25; U^0 = f
    const float lambda = 1.0f, step = 0.25f;
    wmc::TileParams tp{};
    tp.u = f;
    tp.f = f;
    tp.out = u;
    tp.ld = ld;
    tp.ld_out = ld;
    tp.h = h;
    tp.w = w;
    tp.use_tma = 1;
    tp.c_keep = 1.0f - step;
    tp.c_f = step;
    tp.c_h = step * lambda / 12.0f;
    tp.status = status;
    tp.pdl = 0;
    tp.f_tma = 1;
    tp.flags = flags;
    tp.flag_wait = 1;  // a launch number no launch stores
    tp.flag_set = 1;
    e = launch_tile(WMC_F32, WMC_BOUNDARY_REPLICATE, kDefaultTile, 4, maps, tp, -1, st);
    if (e != cudaSuccess) return cuda_fail(e, "flow kernel launch");
    return WMC_OK;
}

size_t wmc_backward_workspace_size(int32_t n, int32_t h, int32_t w, int64_t ld, int32_t K,
                                   int32_t ckpt_every) {
    const size_t base = wmc_unrolled_workspace_size(n, h, w, ld, K, ckpt_every);
    if (base == 0) return 0;
    // the unrolled workspace, then U^K of the stack (the forward's output, not returned)
    return round_up(base, WMC_WORKSPACE_ALIGN) +
           round_up(span_bytes(n * h, w, ld, sizeof(float)), WMC_WORKSPACE_ALIGN);
}

wmc_status_t wmc_backward(const float *f, const float *lambda, float step, int32_t K,
                          int32_t ckpt_every, int32_t n, int32_t h, int32_t w, int64_t ld,
                          wmc_boundary_t bnd, const float *grad_u, float *grad_f,
                          float *grad_lambda, void *workspace, size_t workspace_bytes,
                          wmc_stream_t stream) {
    g_last_error[0] = 0;
    wmc_status_t s = check_unrolled(f, lambda, step, K, ckpt_every, n, h, w, ld, bnd);
    if (s != WMC_OK) return s;
    if ((int64_t)n * h > 0x7fffffffLL) return fail(WMC_ERR_INVALID_ARG, "n * h beyond 2^31 - 1");
    const size_t need = wmc_backward_workspace_size(n, h, w, ld, K, ckpt_every);
    if (!workspace || workspace_bytes < need)
        return fail(WMC_ERR_WORKSPACE, "workspace of %zu bytes needed, %zu given", need,
                    workspace ? workspace_bytes : (size_t)0);
    if ((uintptr_t)workspace % WMC_WORKSPACE_ALIGN)
        return fail(WMC_ERR_WORKSPACE, "workspace not %d-byte aligned", WMC_WORKSPACE_ALIGN);
    const size_t nbytes = span_bytes(n * h, w, ld, sizeof(float));
    if (overlap(workspace, need, f, nbytes) || overlap(workspace, need, grad_u, nbytes) ||
        (grad_f && overlap(workspace, need, grad_f, nbytes)))
        return fail(WMC_ERR_ALIAS, "workspace overlaps f, grad_u or grad_f");
    const size_t inner = round_up(wmc_unrolled_workspace_size(n, h, w, ld, K, ckpt_every), WMC_WORKSPACE_ALIGN);
    float *uK = reinterpret_cast<float *>(static_cast<char *>(workspace) + inner);
    // the forward sweep stores the checkpoints in the inner workspace; the reverse sweep reads them
    s = wmc_unrolled_forward(f, lambda, step, K, ckpt_every, n, h, w, ld, bnd, uK, workspace, inner, stream);
    if (s != WMC_OK) return s;
    return wmc_unrolled_backward(f, lambda, step, K, ckpt_every, n, h, w, ld, bnd, grad_u, grad_f,
                                 grad_lambda, workspace, inner, stream);
}

}  // extern "C"
