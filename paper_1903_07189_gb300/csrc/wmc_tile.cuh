// wmc_tile.cuh -- temporally blocked WMC flow kernel: T Jacobi steps per launch in shared memory,
// for one image or for a batch of images of different sizes in the same launch.
//
// The update U^{t+1} = U^t + step (lambda H^w(U^t) - mu (U^t - f)) (Sec. V-B, Eq. MCF) is
// Jacobi-ordered: every pixel of step t+1 reads only U^t.  So a CTA can load a window of U^t,
// take T steps on it without talking to anyone, and write back the part of the window that is
// still exact: each step's stale border moves one cell inwards.
//
// Geometry (element coordinates; X0, Y0 = global position of shared cell (0,0)):
//   loaded window  [X0, X0+LW) x [Y0, Y0+LH)       one 2-D TMA box, zero-filled outside the image
//   updated cells  [X0+2+d, X0+2+d+CW) x [Y0+1, Y0+1+CH)    every step (CW = 128, CH = 64)
//   exact after T  [X0+1+d+T, X0+3+d+CW-T) x [Y0+T, Y0+2+CH-T)
//   written back   [x0, x0+OWt) x [y0, y0+OHt),  X0 = x0 - (T+1) rounded down to the TMA
//                  alignment (16 bytes of elements), d = x0 - (T+1) - X0, y0 = Y0 + T
// The output tile size (OWt, OHt) is a launch parameter: a single-image launch uses the largest
// exact tile of its T (Out<S,T>); a batch uses the tile of its deepest T for every launch, which
// any shallower launch also covers exactly (its exact region is larger), so one tile table
// serves them all.
// Each tile rounds its own window origin down to the TMA alignment, which keeps every TMA
// x-coordinate aligned without constraining where output tiles start.
//
// Threads: 16 warps as 2 (x) x 8 (y); lane l of warp (wx, wy) updates columns j = 2 + d + 64 wx + l
// and j + 32 for rows i = 1 + 8 wy .. 8 + 8 wy.  The two columns are the two lanes of packed
// FP32x2 arithmetic: every operand pair (west, centre, east neighbours of both cells) is read
// by two conflict-free 4-byte shared loads straight into an aligned register pair, so no
// register shuffling is needed (pairing the adjacent columns j, j+1 instead would make six of
// the nine operands straddle register pairs).  Offsets are constants: the inner loop has no index
// arithmetic and no per-cell predicates in tiles that lie inside the image.
//
// Image boundary.  ZERO: the TMA fill supplies the zeros; in tiles touching the border, cells
// outside the image are rewritten as 0 every step.  REPLICATE: the ring of cells just outside
// the image is kept equal to its nearest in-image cell (refreshed after the load and after every
// step, in tiles touching the border only), so in-image cells read their neighbours without any
// clamping and produce exactly what clamped reads would.  Warps whose cells all lie beyond that
// ring (tiles overhanging the image) skip the arithmetic: no in-image cell reads those cells.
//
// The update's f term (c_f f, constant over the T steps) sits in registers, 8 rows x 2 columns
// per thread.  For FP32 storage f's window comes as a second TMA box with the same origin, into a
// third shared buffer, completing the same mbarrier (f is never written by a flow launch, so its
// copy is issued before the wait for the previous launch); 16-bit storage reads f with
// predicated plain loads.
//
// Shared memory always holds FP32; for BF16/FP16 storage the TMA box lands in a staging area
// and is widened once, and every step rounds its result to the storage type, so the arithmetic
// is identical to the single-step streaming kernel.
//
// Batches: a tile table lists (image, x0, y0) for every tile of every image; each image has a
// descriptor with its buffers (f, u, workspace), pitch, size, update coefficients (its own
// lambda and step) and one tensor map per buffer.  A launch reads every image from the buffer of
// one role and writes the buffer of another, so all images advance T steps together.
#pragma once

#include <cuda.h>
#include <string.h>

#include <algorithm>
#include <atomic>

#include "wmc_device.cuh"
#include "wmc_internal.h"

namespace wmc {

constexpr int kCW = 128;   // updated columns per step
constexpr int kCH = 64;    // updated rows per step
constexpr int kRY = 8;     // rows per thread
constexpr int kTileWX = 2; // warps across (64 columns each)
constexpr int kTileWY = kCH / kRY;  // warps down
constexpr int kTileThreadsV2 = 32 * kTileWX * kTileWY;  // 512
#ifndef WMC_TILE_MIN_BLOCKS
#define WMC_TILE_MIN_BLOCKS 2  // CTAs per SM the register allocation must allow (1 CTA/SM with
                               // 82 registers measured 20% slower at 4096^2)
#endif

template <typename S> struct Geom {
    static constexpr int A = 16 / (int)sizeof(S);                 // TMA x alignment (elements)
    // loaded width: the updated columns start 2 + d into the window (d < A, below) and their
    // east neighbours reach column 130 + d
    static constexpr int LW = ((kCW + 2 + A + A - 1) / A) * A;
    static constexpr int LH = kCH + 2;                            // loaded height
    static constexpr int P = LW;                                  // shared pitch (floats)
    static constexpr int BUF = LH * P;                            // floats per buffer
    static constexpr int STAGE_BYTES = sizeof(S) == 4 ? 0 : LH * LW * (int)sizeof(S);
    // FP32 storage: the window of f arrives by TMA too, into a third buffer after the two
    // ping-pong buffers (16-bit storage reads f with plain loads)
    static constexpr int F_BYTES = sizeof(S) == 4 ? BUF * 4 : 0;
    static constexpr int SMEM = 2 * BUF * 4 + STAGE_BYTES + F_BYTES + 128;  // + alignment slack
    static_assert(sizeof(S) != 4 || (2 * BUF * 4) % 128 == 0, "the f window must start 128-byte aligned");
};

// Output tile of a T-step single-image launch, width OW and height OH.  The window origin is the
// output origin x0 less T + 1, rounded down to the TMA alignment A (window_x0); the d = 0..A-1
// columns lost to the rounding shift the updated columns (2 + d .. 129 + d in the window), so
// after T steps the window is exact on exactly [x0, x0 + CW + 2 - 2T).  Rows: y0 - T.
template <typename S, int T> struct Out {
    static constexpr int OW = kCW + 2 - 2 * T;
    static constexpr int OH = kCH + 2 - 2 * T;
};

template <typename S, int T>
__host__ __device__ __forceinline__ int window_x0(int x0) {
    return (x0 - (T + 1)) & ~(Geom<S>::A - 1);  // floor to a multiple of A (also below 0)
}

// One image of a batch (device memory; 64-byte aligned for the tensor maps).
struct alignas(64) BatchImage {
    CUtensorMap map[3];   // tensor maps over buf[0..2]
    const void *buf[3];   // 0: f (read only), 1: u (output), 2: workspace image
    int64_t ld;
    int32_t h, w;
    float c_keep, c_f, c_h;
    int32_t use_tma[3];
};

struct TileV2Params {
    // single image (tiles from blockIdx)
    const void *u;    // U^t (device); read through the tensor map when use_tma
    const void *f;    // f or nullptr (mean-curvature flow)
    void *out;        // U^{t+T}
    int64_t ld;       // pitch of u, f and out
    int32_t h, w;
    int32_t ntx;      // tiles per row of tiles
    int32_t use_tma;
    float c_keep, c_f, c_h;
    // batch (tiles from the table)
    const BatchImage *images;
    const int4 *tiles;    // (image, x0, y0, 0) per tile
    int32_t src_role, dst_role;
    // both
    int32_t owt, oht;     // output tile size
    unsigned int *status; // device status word (bit 0: a bounded wait gave up) or nullptr
    int32_t pdl;          // host side: launch as a programmatic dependent of the previous launch
    int32_t f_tma;        // single image, FP32: f is read through the second tensor map
};

// Programmatic dependent launch: a launch made with the programmatic-serialization attribute may
// start while the previous kernel in the stream finishes (its CTAs fill the SMs the last wave
// leaves idle and do their set-up); griddep_wait() then blocks until that kernel has completed
// and its writes are visible.  Both are no-ops for a launch made without the attribute.
__device__ __forceinline__ void griddep_launch_dependents() {
    asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
}
__device__ __forceinline__ void griddep_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }

// ------------------------------------------------------------------ TMA / mbarrier helpers
__device__ __forceinline__ uint32_t smem_u32(const void *p) {
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ uint64_t global_timer_ns() {
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

__device__ __forceinline__ void mbar_init(uint32_t bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

__device__ __forceinline__ void mbar_expect_tx(uint32_t bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes)
                 : "memory");
}

// Orders this thread's (and, after a CTA barrier, the CTA's) earlier shared-memory accesses of
// the generic proxy before later async-proxy (TMA) accesses of the same memory: issued before a
// TMA copy refills a buffer that threads have been reading.
__device__ __forceinline__ void fence_proxy_async_smem() {
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

__device__ __forceinline__ void tma_load_2d(uint32_t dst, const CUtensorMap *map, int x, int y,
                                            uint32_t bar) {
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.tile.mbarrier::complete_tx::bytes"
        " [%0], [%1, {%2, %3}], [%4];" ::"r"(dst),
        "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(bar)
        : "memory");
}

// Wait for the barrier's phase; give up after `limit_ns` (returns false).  Each try_wait may
// suspend the thread in hardware for up to 1 ms, so the loop spins very little.
__device__ __forceinline__ bool mbar_wait_bounded(uint32_t bar, uint32_t phase, uint64_t limit_ns) {
    const uint64_t t0 = global_timer_ns();
    for (;;) {
        uint32_t done;
        asm volatile(
            "{ .reg .pred p; mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2, %3;"
            " selp.u32 %0, 1, 0, p; }"
            : "=r"(done)
            : "r"(bar), "r"(phase), "r"(1000000u)
            : "memory");
        if (done) return true;
        if (global_timer_ns() - t0 > limit_ns) return false;
    }
}

constexpr uint64_t kWaitLimitNs = 200ull * 1000 * 1000;  // 0.2 s

// ------------------------------------------------------------------------------- kernel
// Per-thread constants of one tile.
struct TileCtx {
    int j, ib;         // shared column of the thread's first cell (second: j + 32), first row
    int X0, Y0, gx;    // window origin, image column of the first cell
    int h, w;
    bool cin0, cin1;   // the two cells' columns lie inside the image
    bool out0, out1;   // ... and inside the output tile
    unsigned out_rows; // bit k: row ib + k is an output row inside the image
    float c_keep, c_h;
};

enum StepWrite { WRITE_INTERIOR = 0, WRITE_BORDER = 1, WRITE_GLOBAL = 2 };

// Columns j-1, j, j+1 of one shared row for both lanes (j and j+32) as aligned pairs.
struct Row3 {
    float2 w, c, e;
};
__device__ __forceinline__ Row3 load_row3(const float *r) {
    Row3 o;
    o.w = make_float2(r[-1], r[31]);
    o.c = make_float2(r[0], r[32]);
    o.e = make_float2(r[1], r[33]);
    return o;
}

// One Jacobi step over the thread's kRY rows x 2 columns, reading `src`, writing `dst` (shared)
// or the output image (last step).
template <int WMODE, typename S, int BND>
__device__ __forceinline__ void tile_step(const float *__restrict__ src, float *__restrict__ dst,
                                          const TileCtx &c, const float2 (&g)[kRY],
                                          S *__restrict__ orow = nullptr, int64_t ld = 0) {
    using G = Geom<S>;
    constexpr int P = G::P, LH = G::LH, LW = G::LW;
    const float2 ch = make_float2(c.c_h, c.c_h), ck = make_float2(c.c_keep, c.c_keep);
    const float *rp = src + (c.ib - 1) * P + c.j;
    Row3 r0 = load_row3(rp), r1 = load_row3(rp + P);
#pragma unroll
    for (int k = 0; k < kRY; ++k) {
        const Row3 r2 = load_row3(rp + (k + 2) * P);
        const float2 hw = half_laplace12_x2(r0.w, r0.c, r0.e, r1.w, r1.c, r1.e, r2.w, r2.c, r2.e);
        float2 v = __ffma2_rn(ch, hw, __ffma2_rn(ck, r1.c, g[k]));
        const int i = c.ib + k;
        if (WMODE == WRITE_INTERIOR) {
            const float2 rv = Store<S>::round2(v);
            float *d = dst + i * P + c.j;
            d[0] = rv.x;
            d[32] = rv.y;
        } else if (WMODE == WRITE_BORDER) {
            // tiles touching the border: cells outside the image keep 0 (ZERO) or are left
            // for the ring refresh after the step (REPLICATE)
            const int gy = c.Y0 + i;
            const bool rin = (gy >= 0) & (gy < c.h);
            const bool in0 = rin & c.cin0, in1 = rin & c.cin1;
            float *d = dst + i * P + c.j;
            const float2 rv = Store<S>::round2(v);
            if (BND == BND_ZERO) {
                d[0] = in0 ? rv.x : 0.0f;
                d[32] = in1 ? rv.y : 0.0f;
            } else {
                if (in0) d[0] = rv.x;
                if (in1) d[32] = rv.y;
            }
        } else {
            // predicated stores, no branch: row Y0 + ib + k, columns gx and gx + 32
            const bool rk = (c.out_rows >> k) & 1u;
            S *o = orow + (int64_t)k * ld;
            if (rk & c.out0) Store<S>::store(o, v.x);
            if (rk & c.out1) Store<S>::store(o + 32, v.y);
        }
        r0 = r1;
        r1 = r2;
    }
}

// REPLICATE: set the ring of cells just outside the image (image rows -1 and h, image columns -1
// and w, where they cross the window) to the value of the nearest in-image cell, so that in-image
// cells can read their neighbours without clamping.  Corner cells belong to two segments and get
// the same value from both.
template <typename S>
__device__ __forceinline__ void refresh_ring(float *buf, int X0, int Y0, int h, int w, int tid) {
    using G = Geom<S>;
    constexpr int LW = G::LW, LH = G::LH, P = G::P;
    const int ir0 = -1 - Y0, ir1 = h - Y0;  // shared rows of image rows -1 and h
    const int jc0 = -1 - X0, jc1 = w - X0;  // shared columns of image columns -1 and w
    const int jlo = max(jc0, 0), jhi = min(jc1, LW - 1);
    const int ilo = max(ir0, 0), ihi = min(ir1, LH - 1);
    for (int t = tid; t < 2 * (LW + LH); t += kTileThreadsV2) {
        int i, j2;
        if (t < 2 * LW) {
            i = (t < LW) ? ir0 : ir1;
            j2 = (t < LW) ? t : t - LW;
            if (i < 0 || i >= LH || j2 < jlo || j2 > jhi) continue;
        } else {
            const int q = t - 2 * LW;
            j2 = (q < LH) ? jc0 : jc1;
            i = (q < LH) ? q : q - LH;
            if (j2 < 0 || j2 >= LW || i < ilo || i > ihi) continue;
        }
        const int yy = Y0 + i, xx = X0 + j2;
        const int ci = min(max(yy, 0), h - 1) - Y0, cj = min(max(xx, 0), w - 1) - X0;
        buf[i * P + j2] = buf[ci * P + cj];
    }
}

// One tile's job: which image buffers, coefficients and output tile.
template <typename S> struct TileJob {
    const S *u;                // U^t (read through `map` when use_tma)
    const S *f;                // f or nullptr
    const CUtensorMap *map;
    const CUtensorMap *fmap;   // f's tensor map, used when f_tma
    bool f_tma;                // FP32 and TMA: f's window is loaded with U's into fbuf
    int64_t ld;
    int h, w;
    float c_keep, c_h, c_f;
    int x0, y0;                // output tile origin
    bool use_tma;
};

// Everything a CTA does for one tile: load the window of U^t, take T steps in shared memory and
// write the output tile through `out_of()` (called after the steps, so the output pointer is not
// kept in registers through them).  `phase` is the mbarrier parity this tile's load completes.
// Returns false if the window load timed out (the status word is set).
template <int T, typename S, int BND, typename OutFn>
__device__ __forceinline__ bool tile_job(const TileJob<S> &jb, int owt, int oht,
                                         unsigned int *status, float *buf0, float *buf1,
                                         uint64_t *bar, uint32_t phase, OutFn out_of) {
    using G = Geom<S>;
    constexpr int LW = G::LW, LH = G::LH, BUF = G::BUF;
    TileCtx c;
    c.h = jb.h;
    c.w = jb.w;
    c.c_keep = jb.c_keep;
    c.c_h = jb.c_h;
    const int h = c.h, w = c.w;
    const int x0 = jb.x0, y0 = jb.y0;
    const int X0 = window_x0<S, T>(x0), Y0 = y0 - T;
    const int tid = threadIdx.x;
    const bool border = (X0 < 0) | (Y0 < 0) | (X0 + LW > w) | (Y0 + LH > h);

    // ---- issue the load of the window of U^t (thread 0 alone owns the barrier: it issues the
    // copy and later waits for it, so the other threads never poll it).  U^t is the previous
    // launch's output: wait for that launch first (every later access of this CTA to U^t or to
    // the output buffer comes after this thread's wait through the CTA barriers below).
    // FP32 with TMA: f's window (same box and origin as U's) lands in the third buffer and
    // completes the same barrier.  f is never written by a flow launch, so its copy goes out
    // before the wait for the previous launch.
    const bool ftma = sizeof(S) == 4 && jb.use_tma && jb.f_tma && jb.f != nullptr;
    float *fbuf = buf1 + BUF;
    if (jb.use_tma) {
        if (tid == 0) {
            mbar_expect_tx(smem_u32(bar), (uint32_t)(LW * LH * sizeof(S)) * (ftma ? 2u : 1u));
            if (ftma) tma_load_2d(smem_u32(fbuf), jb.fmap, X0, Y0, smem_u32(bar));
            griddep_wait();
            void *dst = (sizeof(S) == 4) ? static_cast<void *>(buf0)
                                         : static_cast<void *>(buf1 + BUF);  // staging
            tma_load_2d(smem_u32(dst), jb.map, X0, Y0, smem_u32(bar));
        }
    } else {
        constexpr int P = G::P;
        griddep_wait();
        for (int idx = tid; idx < LH * LW; idx += kTileThreadsV2) {
            const int i = idx / LW, j = idx - (idx / LW) * LW;
            const int gy = Y0 + i, gx = X0 + j;
            float v = 0.0f;
            if (gy >= 0 && gy < h && gx >= 0 && gx < w) v = Store<S>::load(jb.u + (int64_t)gy * jb.ld + gx);
            buf0[i * P + j] = v;
        }
    }

    // ---- per-thread geometry and f (overlaps the load)
    const int lane = tid & 31, warp = tid >> 5;
    c.j = 2 + (x0 - (T + 1) - X0) + 64 * (warp & 1) + lane;  // shifted by the rounding d
    c.ib = 1 + kRY * (warp >> 1);
    c.X0 = X0;
    c.Y0 = Y0;
    c.gx = X0 + c.j;
    c.cin0 = (c.gx >= 0) & (c.gx < w);
    c.cin1 = (c.gx + 32 >= 0) & (c.gx + 32 < w);
    c.out0 = c.cin0 & (c.gx >= x0) & (c.gx < x0 + owt);
    c.out1 = c.cin1 & (c.gx + 32 >= x0) & (c.gx + 32 < x0 + owt);
    // bit k of in_rows: image row Y0 + ib + k exists; of out_rows: it is also an output row.
    // Both are contiguous ranges of the thread's kRY rows.
    auto row_range = [](int lo, int hi) -> unsigned {  // bits [max(lo,0), min(hi,kRY))
        lo = max(lo, 0);
        hi = min(hi, kRY);
        return hi > lo ? ((1u << hi) - 1u) & ~((1u << lo) - 1u) : 0u;
    };
    const int r0 = Y0 + c.ib;
    const unsigned in_rows = row_range(-r0, h - r0);
    c.out_rows = in_rows & row_range(y0 - r0, y0 + oht - r0);
    float2 g[kRY];
    const float2 cf = make_float2(jb.c_f, jb.c_f);
    if (!ftma) {
        const S *fr = jb.f + (int64_t)(Y0 + c.ib) * jb.ld + c.gx;
        const bool hasf = jb.f != nullptr;
#pragma unroll
        for (int k = 0; k < kRY; ++k) {
            // predicated loads, no branch
            const bool rk = hasf & ((in_rows >> k) & 1u);
            const S *fk = fr + (int64_t)k * jb.ld;
            const float a = (rk & c.cin0) ? Store<S>::load(fk) : 0.0f;
            const float b = (rk & c.cin1) ? Store<S>::load(fk + 32) : 0.0f;
            g[k] = __fmul2_rn(cf, make_float2(a, b));
        }
    }

    // ---- wait for the window: thread 0 waits on the barrier (its completion makes the copied
    // data visible to it), then the CTA barrier orders everyone else's reads after that
    if (jb.use_tma) {
        const bool ok = (tid != 0) || mbar_wait_bounded(smem_u32(bar), phase, kWaitLimitNs);
        if (__syncthreads_or(!ok)) {
            if (tid == 0 && status) atomicOr(status, 1u);
            return false;
        }
        if constexpr (sizeof(S) != 4) {  // widen the staged 16-bit box, 8 elements per 16-byte access
            static_assert((LH * LW) % 8 == 0, "the staged box is a whole number of 16-byte chunks");
            const uint4 *stage = reinterpret_cast<const uint4 *>(buf1 + BUF);
            float4 *dst4 = reinterpret_cast<float4 *>(buf0);
            for (int q = tid; q < LH * LW / 8; q += kTileThreadsV2) {
                const uint4 raw = stage[q];
                const float2 a = Store<S>::unpack2(raw.x), b = Store<S>::unpack2(raw.y);
                const float2 c2 = Store<S>::unpack2(raw.z), d2 = Store<S>::unpack2(raw.w);
                dst4[2 * q] = make_float4(a.x, a.y, b.x, b.y);
                dst4[2 * q + 1] = make_float4(c2.x, c2.y, d2.x, d2.y);
            }
            __syncthreads();
        }
    } else {
        __syncthreads();
    }
    if (ftma) {  // f as loaded by TMA: zero outside the image, like the plain loads' predicates
        const float *fr = fbuf + c.ib * G::P + c.j;
#pragma unroll
        for (int k = 0; k < kRY; ++k) g[k] = __fmul2_rn(cf, make_float2(fr[k * G::P], fr[k * G::P + 32]));
    }

    // ---- REPLICATE: fill the ring just outside the image from its nearest in-image cell.
    if (BND == BND_REPLICATE && border) {
        refresh_ring<S>(buf0, X0, Y0, h, w, tid);
        __syncthreads();
    }

    // ---- T steps: ping-pong buf0 -> buf1 -> buf0 ...; the last one writes the output tile.
    // A warp whose cells all lie beyond the ring just outside the image (rows >= h + 1, or
    // columns >= w + 1: tiles that overhang the image's bottom or right edge) has nothing that
    // any in-image cell reads, so it skips the arithmetic (it still takes part in the barriers).
    const bool idle = (Y0 + c.ib >= h + 1) | (c.gx - lane >= w + 1);
#pragma unroll 1
    for (int s = 0; s < T - 1; ++s) {
        const float *src = (s & 1) ? buf1 : buf0;
        float *dst = (s & 1) ? buf0 : buf1;
        if (!border) {
            tile_step<WRITE_INTERIOR, S, BND>(src, dst, c, g);
            __syncthreads();
        } else {
            if (!idle) tile_step<WRITE_BORDER, S, BND>(src, dst, c, g);
            __syncthreads();
            if (BND == BND_REPLICATE) {
                refresh_ring<S>(dst, X0, Y0, h, w, tid);
                __syncthreads();
            }
        }
    }
    if (idle) return true;  // none of its cells is an output cell inside the image
    int64_t ldo;
    S *out = out_of(&ldo);
    tile_step<WRITE_GLOBAL, S, BND>(((T - 1) & 1) ? buf1 : buf0, nullptr, c, g,
                                    out + (int64_t)(Y0 + c.ib) * ldo + c.gx, ldo);
    return true;
}

template <int T, typename S, int BND, bool BATCH>
__global__ void __launch_bounds__(kTileThreadsV2, WMC_TILE_MIN_BLOCKS)
    tile_v2_kernel(const __grid_constant__ CUtensorMap tmap, const __grid_constant__ CUtensorMap fmap,
                   const TileV2Params p) {
    extern __shared__ unsigned char smem_raw[];
    __shared__ __align__(8) uint64_t bar;
    // 128-byte aligned start of the buffers, formed as an offset into the __shared__ array (not
    // through an integer cast) so that every access below stays a shared-memory access
    float *buf0 = reinterpret_cast<float *>(smem_raw + ((128u - (smem_u32(smem_raw) & 127u)) & 127u));
    float *buf1 = buf0 + Geom<S>::BUF;

    // ---- this CTA's job: image, buffers, coefficients and output tile
    TileJob<S> jb;
    if (BATCH) {
        const int4 t = p.tiles[blockIdx.x];
        const BatchImage &im = p.images[t.x];
        jb.u = static_cast<const S *>(im.buf[p.src_role]);
        jb.f = static_cast<const S *>(im.buf[0]);
        jb.ld = im.ld;
        jb.h = im.h;
        jb.w = im.w;
        jb.c_keep = im.c_keep;
        jb.c_h = im.c_h;
        jb.c_f = im.c_f;
        jb.map = &im.map[p.src_role];
        jb.use_tma = im.use_tma[p.src_role] != 0;
        jb.fmap = &im.map[0];
        jb.f_tma = im.use_tma[0] != 0;
        jb.x0 = t.y;
        jb.y0 = t.z;
    } else {
        jb.u = static_cast<const S *>(p.u);
        jb.f = static_cast<const S *>(p.f);
        jb.ld = p.ld;
        jb.h = p.h;
        jb.w = p.w;
        jb.c_keep = p.c_keep;
        jb.c_h = p.c_h;
        jb.c_f = p.c_f;
        jb.map = &tmap;
        jb.use_tma = p.use_tma != 0;
        jb.fmap = &fmap;
        jb.f_tma = p.f_tma != 0;
        const int ty = blockIdx.x / p.ntx, tx = blockIdx.x - ty * p.ntx;
        jb.x0 = tx * p.owt;
        jb.y0 = ty * p.oht;
    }
    // the next launch may be scheduled once every CTA of this one is running
    griddep_launch_dependents();
    if (jb.use_tma && threadIdx.x == 0) mbar_init(smem_u32(&bar), 1);
    // the output pointer is looked up again after the steps (kernel parameters, or the image
    // descriptor in L1) rather than kept in registers through them
    tile_job<T, S, BND>(jb, p.owt, p.oht, p.status, buf0, buf1, &bar, 0u, [&](int64_t *ldo) -> S * {
        if (BATCH) {
            const BatchImage &im = p.images[p.tiles[blockIdx.x].x];
            *ldo = im.ld;
            return static_cast<S *>(const_cast<void *>(im.buf[p.dst_role]));
        }
        *ldo = p.ld;
        return static_cast<S *>(p.out);
    });
}

template <int T, typename S, int BND, bool BATCH>
cudaError_t launch_tile_v2_t(const CUtensorMap *map, TileV2Params p, int64_t nblocks,
                             cudaStream_t st) {
    using G = Geom<S>;
    if (!BATCH) {
        p.owt = Out<S, T>::OW;
        p.oht = Out<S, T>::OH;
        const int64_t ntx = (p.w + p.owt - 1) / p.owt, nty = (p.h + p.oht - 1) / p.oht;
        nblocks = ntx * nty;
        p.ntx = (int32_t)ntx;
    }
    if (nblocks > 0x7fffffffLL) return cudaErrorInvalidConfiguration;
    if (nblocks == 0) return cudaSuccess;
    // The shared-memory opt-in is per device; set it once per device so that launches made
    // while a stream is being captured into a graph issue no attribute calls.
    static std::atomic<uint64_t> attr_set{0};
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    const uint64_t bit = 1ull << (dev & 63);
    if (!(attr_set.load(std::memory_order_acquire) & bit)) {
        e = cudaFuncSetAttribute(tile_v2_kernel<T, S, BND, BATCH>,
                                 cudaFuncAttributeMaxDynamicSharedMemorySize, G::SMEM);
        if (e != cudaSuccess) return e;
        attr_set.fetch_or(bit, std::memory_order_release);
    }
    // map: the tensor maps of U and of f (single image; f's is read only when p.f_tma)
    alignas(64) CUtensorMap dummy[2];
    if (BATCH || !p.use_tma) {
        memset(dummy, 0, sizeof dummy);
        map = dummy;
        p.f_tma = 0;
    }
    if (!p.pdl) {
        tile_v2_kernel<T, S, BND, BATCH><<<(unsigned)nblocks, kTileThreadsV2, G::SMEM, st>>>(map[0], map[1], p);
        return cudaGetLastError();
    }
    cudaLaunchConfig_t cfg{};
    cfg.gridDim = dim3((unsigned)nblocks);
    cfg.blockDim = dim3(kTileThreadsV2);
    cfg.dynamicSmemBytes = G::SMEM;
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, tile_v2_kernel<T, S, BND, BATCH>, map[0], map[1], p);
}

template <typename S, int BND>
cudaError_t launch_tile_v2_steps(int steps, const CUtensorMap *map, const TileV2Params &p,
                                 int64_t batch_tiles, cudaStream_t st) {
    const bool b = batch_tiles >= 0;
#define WMC_TILE_CASE(T)                                                                        \
    case T:                                                                                     \
        return b ? launch_tile_v2_t<T, S, BND, true>(map, p, batch_tiles, st)                   \
                 : launch_tile_v2_t<T, S, BND, false>(map, p, 0, st);
    switch (steps) {
        WMC_TILE_CASE(1)
        WMC_TILE_CASE(2)
        WMC_TILE_CASE(3)
        WMC_TILE_CASE(4)
        WMC_TILE_CASE(5)
        WMC_TILE_CASE(6)
        WMC_TILE_CASE(7)
        WMC_TILE_CASE(8)
        default: return cudaErrorInvalidValue;
    }
#undef WMC_TILE_CASE
}

}  // namespace wmc
