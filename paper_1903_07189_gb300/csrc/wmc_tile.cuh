// wmc_tile.cuh -- temporally blocked WMC flow kernel: T Jacobi steps per launch in shared memory,
// for one image or for a batch of images of different sizes in the same launch.
//
// The update U^{t+1} = U^t + step (lambda H^w(U^t) - mu (U^t - f)) (Sec. V-B, Eq. MCF) is
// Jacobi-ordered: every pixel of step t+1 reads only U^t.  So a CTA can load a window of U^t,
// take T steps on it without talking to anyone, and write back the part of the window that is
// still exact: each step's stale border moves one cell inwards.
//
// Geometry (element coordinates; X0, Y0 = global position of shared cell (0,0)).  A CTA of NW
// warps updates 128 columns x CH = 4 NW rows every step (NW = 16: 128 x 64; NW = 8: 128 x 32,
// the shape for small or short images):
//   loaded window  [X0, X0+LW) x [Y0, Y0+CH+2)       one 2-D TMA box, zero-filled outside the image
//   updated cells  [X0+2+d, X0+130+d) x [Y0+1, Y0+1+CH)    every step
//   exact after T  [X0+1+d+T, X0+131+d-T) x [Y0+T, Y0+2+CH-T)
//   written back   [x0, x0+OWt) x [y0, y0+OHt),  X0 = x0 - (T+1) rounded down to the TMA
//                  alignment (16 bytes of elements), d = x0 - (T+1) - X0, y0 = Y0 + T
// A single-image launch uses the largest exact output tile of its T (130 - 2T by CH + 2 - 2T); a
// batch uses the tile of its deepest T for every launch, which any shallower launch also covers
// exactly (its exact region is larger), so one tile table serves them all.
// Each tile rounds its own window origin down to the TMA alignment, which keeps every TMA
// x-coordinate aligned without constraining where output tiles start.
//
// Threads: warps as 2 (x) x NW/2 (y); lane l of warp (wx, wy) updates columns j = 2 + d + 64 wx + l
// and j + 32 for rows i = 1 + 8 wy .. 8 + 8 wy.  The two columns are the two lanes of packed
// FP32x2 arithmetic: every operand pair (west, centre, east neighbours of both cells) is read
// by two conflict-free 4-byte shared loads straight into an aligned register pair, so no
// register moves are needed (pairing the adjacent columns j, j+1 instead would make six of
// the nine operands straddle register pairs; four adjacent columns per lane, read with one
// 16-byte load, were measured slower: the register moves that form their pairs cost more than
// the loads they save).  Offsets are constants: the inner loop has no index arithmetic and no
// per-cell predicates in tiles that lie inside the image.
//
// Image boundary.  ZERO: the TMA fill supplies the zeros; in tiles touching the border, cells
// outside the image are rewritten as 0 every step.  REPLICATE: the ring of cells just outside
// the image is kept equal to its nearest in-image cell (refreshed once after the load; after each
// step the ring-column cells are computed at their source columns and the ring rows stored by the
// edge rows' threads, in tiles touching the border only), so in-image cells read their
// neighbours without any clamping and produce exactly what clamped reads would.  Warps whose
// cells all lie beyond that
// ring (tiles overhanging the image) skip the arithmetic: no in-image cell reads those cells.
//
// The update's f term (c_f f, constant over the T steps) sits in registers, 8 rows x 2 columns
// per thread.  f's window comes as a second TMA box with the same origin (FP32: into a third
// shared buffer; 16-bit storage: into buffer 1, whose first write comes after f has been read),
// completing the same mbarrier; f is never written by a flow launch, so its copy is issued before
// the wait for the previous launch.  Without TMA (pitches TMA cannot describe) f is read with
// predicated plain loads.
//
// Shared memory always holds FP32 for the steps; for BF16/FP16 storage the TMA box of U lands
// in a staging area and is widened once, and every step rounds its result to the storage type,
// so the arithmetic is identical to the single-step streaming kernel.
//
// Batches: a tile table lists (image, x0, y0) for every tile of every image; each image has a
// descriptor with its buffers (f, u, two workspace images), pitches, size, update coefficients
// (its own lambda and step) and one tensor map per buffer it reads.  A launch reads every image
// from the buffer of one role and writes the buffer of another, so all images advance T steps
// together; the launches between the first and the last ping-pong between the two workspace
// images, so every buffer read has a pitch TMA can describe whatever the caller's pitch.
#pragma once

#include "wmc_window.cuh"

namespace wmc {

// Tile shapes (wmc_config_t.tile): 1 = 16 warps (128 x 64 region), 2 = 8 warps (128 x 32).
__host__ __device__ constexpr int tile_warps(int tile) { return tile == 2 ? 8 : 16; }
constexpr int kQR = 4;  // region rows per warp (CH = kQR * NW)

template <typename S, int NW> struct TGeom {
    static constexpr int THREADS = 32 * NW;
    static constexpr int WY = NW / 2;                 // warps down (2 across)
    static constexpr int CH = kRY * WY;               // updated rows per step
    static constexpr int LH = CH + 2;                 // loaded rows
    static constexpr int LW = Geom<S>::LW;            // loaded columns (elements)
    static constexpr int P = LW;                      // shared pitch (floats)
    static constexpr int BUF = LH * P;                // floats per buffer
    // FP32: f's window in a third buffer after the two ping-pong buffers.  16-bit: U's staged box
    // after them (f's lands in buffer 1)
    static constexpr int EXTRA = sizeof(S) == 4 ? BUF * 4 : LH * LW * (int)sizeof(S);
    static constexpr int SMEM = 2 * BUF * 4 + EXTRA + 128;  // + alignment slack
    static_assert(CH == kQR * NW, "a warp pair covers 8 rows");
    // TMA destinations (buffer 0; FP32: the f window after buffer 1; 16-bit: buffer 1 and the
    // staging area after it) start 128-byte aligned
    static_assert(((sizeof(S) == 4 ? 2 : 1) * BUF * 4) % 128 == 0, "TMA destinations are 128-byte aligned");
    static_assert(LH * LW * (int)sizeof(S) <= BUF * 4, "f's 16-bit window fits in buffer 1");
};

template <typename S, int T>
__host__ __device__ __forceinline__ int window_x0(int x0) {
    return (x0 - (T + 1)) & ~(Geom<S>::A - 1);  // floor to a multiple of A (also below 0)
}

// One image of a batch (device memory; 64-byte aligned for the tensor maps).  Every buffer a
// launch reads (roles 0, 2, 3) has a pitch TMA can describe: when the caller's f does not, the
// plan keeps an aligned copy of it in the workspace, refreshed at the start of every run.
struct alignas(64) BatchImage {
    CUtensorMap map[4];   // tensor maps over buf[0], buf[2], buf[3] (buf[1] is only written)
    const void *buf[4];   // 0: f as read (the caller's f or its copy), 1: u (the caller's output),
                          // 2, 3: workspace ping-pong images
    const void *f_src;    // the caller's f
    int64_t ld;           // pitch of buf[0], buf[2] and buf[3]
    int64_t ld_out;       // pitch of u and f_src (the caller's)
    int32_t h, w;
    float c_keep, c_f, c_h;
    int32_t use_tma[4];
    int32_t copy_f;       // buf[0] is a workspace copy of f_src
};

struct TileParams {
    // single image (tiles from blockIdx)
    const void *u;    // U^t (device); read through the tensor map when use_tma
    const void *f;    // f or nullptr (mean-curvature flow)
    void *out;        // U^{t+T}
    int64_t ld;       // pitch of u and f
    int64_t ld_out;   // pitch of out
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
    int32_t f_tma;        // single image: f is read through the second tensor map
    // single image: per-tile completion flags of this run (one word per tile of this launch's tile
    // grid, zeroed before the run's first launch).  flag_wait > 0: before reading U^t a tile waits
    // until the flags of its 3 x 3 neighbouring tiles are >= flag_wait (the previous launch, same
    // tile grid, has finished those tiles) instead of waiting for the whole previous launch;
    // flag_set > 0: the tile stores flag_set into its own flag once its output is written.
    unsigned int *flags;
    int32_t flag_wait, flag_set;
};

// ------------------------------------------------------------------------------- kernel
// Per-thread constants of one tile.
struct TileCtx {
    int j, ib;         // shared column of the thread's first cell (second: j + 32), first row
    int X0, Y0, gx;    // window origin, image column of the first cell
    int h, w;
    bool cin0, cin1;   // the two cells' columns lie inside the image
    bool out0, out1;   // ... and inside the output tile
    // REPLICATE border tiles: the shared columns the two cells are computed at (their own, or for
    // a cell outside the image the nearest image column's), and whether the cell is stored (its
    // column lies in the image or is the ring column just outside it)
    int jc0, jc1;
    bool st0, st1;
    unsigned out_rows; // bit k: row ib + k is an output row inside the image
    float c_keep, c_h;
};

enum StepWrite { WRITE_INTERIOR = 0, WRITE_BORDER = 1, WRITE_GLOBAL = 2 };

// One Jacobi step over the thread's kRY rows x 2 columns, reading `src`, writing `dst` (shared)
// or the output image (last step).
template <int WMODE, typename S, int BND, int NW>
__device__ __forceinline__ void tile_step(const float *__restrict__ src, float *__restrict__ dst,
                                          const TileCtx &c, const float2 (&g)[kRY],
                                          S *__restrict__ orow = nullptr, int64_t ld = 0) {
    constexpr int P = TGeom<S, NW>::P;
    const float2 ch = make_float2(c.c_h, c.c_h), ck = make_float2(c.c_keep, c.c_keep);
    const float *rp = src + (c.ib - 1) * P + c.j;
    Row3 r0 = load_row3(rp), r1 = load_row3(rp + P);
    // (the rows are unrolled: each row's w + e, w - e and w + e + 2 c are formed once and shared by
    // the three cells that read the row, see half_laplace12_terms)
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
            // tiles touching the border: cells outside the image keep 0 (ZERO)
            const int gy = c.Y0 + i;
            const bool rin = (gy >= 0) & (gy < c.h);
            const bool in0 = rin & c.cin0, in1 = rin & c.cin1;
            float *d = dst + i * P + c.j;
            const float2 rv = Store<S>::round2(v);
            d[0] = in0 ? rv.x : 0.0f;
            d[32] = in1 ? rv.y : 0.0f;
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

// One Jacobi step of a REPLICATE border tile.  The ring just outside the image must hold, after
// every step, the value of the image cell it replicates.  A cell of the ring columns (image column
// -1 or w) is computed at its source column (jc0 / jc1: the same operands, so the same bits as the
// source cell) and stored at its own; the ring rows (image rows -1 and h) are written by the
// threads of image rows 0 and h - 1, which store their two values a row further out as well (a
// warp-uniform branch, taken by one thread row of the tile), the corners included.  Cells of
// other rows and columns outside the image are not stored: no in-image cell reads them.  So no
// refresh pass and no extra CTA barrier separate the steps.
template <typename S, int NW>
__device__ __forceinline__ void tile_step_replicate_border(const float *__restrict__ src,
                                                          float *__restrict__ dst, const TileCtx &c,
                                                          const float2 (&g)[kRY]) {
    constexpr int P = TGeom<S, NW>::P;
    const float2 ch = make_float2(c.c_h, c.c_h), ck = make_float2(c.c_keep, c.c_keep);
    const float *p0 = src + (c.ib - 1) * P + c.jc0, *p1 = src + (c.ib - 1) * P + c.jc1;
    auto row = [&](int r) {
        Row3 o;
        o.w = make_float2(p0[r * P - 1], p1[r * P - 1]);
        o.c = make_float2(p0[r * P], p1[r * P]);
        o.e = make_float2(p0[r * P + 1], p1[r * P + 1]);
        return o;
    };
    Row3 r0 = row(0), r1 = row(1);
    const int top = -c.Y0 - c.ib, bottom = c.h - 1 - c.Y0 - c.ib;  // k of image rows 0 and h - 1
#pragma unroll
    for (int k = 0; k < kRY; ++k) {
        const Row3 r2 = row(k + 2);
        const float2 hw = half_laplace12_x2(r0.w, r0.c, r0.e, r1.w, r1.c, r1.e, r2.w, r2.c, r2.e);
        const float2 rv = Store<S>::round2(__ffma2_rn(ch, hw, __ffma2_rn(ck, r1.c, g[k])));
        const int gy = c.Y0 + c.ib + k;
        float *d = dst + (c.ib + k) * P + c.j;
        if ((gy >= 0) & (gy < c.h)) {
            if (c.st0) d[0] = rv.x;
            if (c.st1) d[32] = rv.y;
        }
        if (k == top) {
            if (c.st0) d[-P] = rv.x;
            if (c.st1) d[32 - P] = rv.y;
        }
        if (k == bottom) {
            if (c.st0) d[P] = rv.x;
            if (c.st1) d[32 + P] = rv.y;
        }
        r0 = r1;
        r1 = r2;
    }
}

// One tile's job: which image buffers, coefficients and output tile.
template <typename S> struct TileJob {
    const S *u;                // U^t (read through `map` when use_tma)
    const S *f;                // f or nullptr
    const CUtensorMap *map;
    const CUtensorMap *fmap;   // f's tensor map, used when f_tma
    bool f_tma;                // f's window is loaded by TMA with U's
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
template <int T, typename S, int BND, int NW, bool UNROLL, typename OutFn, typename DepFn>
__device__ __forceinline__ bool tile_job(const TileJob<S> &jb, int owt, int oht, unsigned int *status,
                                         float *buf0, float *buf1, uint64_t *bar, uint32_t phase,
                                         OutFn out_of, DepFn wait_input) {
    using G = TGeom<S, NW>;
    constexpr int LW = G::LW, LH = G::LH, BUF = G::BUF, P = G::P, NT = G::THREADS;
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
    // launch's output: wait for it first (`wait_input`: the whole previous launch, or the tiles
    // of it that this window reads and this output tile overwrites; every later access of this CTA
    // to U^t or to the output buffer comes after this thread's wait through the CTA barriers
    // below).
    // f's window (same box and origin as U's) completes the same barrier: FP32 into the third
    // buffer, 16-bit storage into buffer 1 (read into registers before the first step writes
    // buffer 1).  f is never written by a flow launch, so its copy goes out before the wait for
    // the previous launch.
    const bool ftma = jb.use_tma && jb.f_tma && jb.f != nullptr;
    void *fwin = (sizeof(S) == 4) ? static_cast<void *>(buf1 + BUF) : static_cast<void *>(buf1);
    void *stage = (sizeof(S) == 4) ? static_cast<void *>(buf0) : static_cast<void *>(buf1 + BUF);
    if (jb.use_tma) {
        if (tid == 0) {
            mbar_expect_tx(smem_u32(bar), (uint32_t)(LW * LH * sizeof(S)) * (ftma ? 2u : 1u));
            wait_input(false);  // per-tile dependencies: before f's copy, which their fence need not wait for
            if (ftma) tma_load_2d(smem_u32(fwin), jb.fmap, X0, Y0, smem_u32(bar));
            wait_input(true);   // the whole previous launch: after f's copy, which then overlaps the wait
            tma_load_2d(smem_u32(stage), jb.map, X0, Y0, smem_u32(bar));
        }
    } else {
        griddep_wait();
        for (int idx = tid; idx < LH * LW; idx += NT) {
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
    if (BND == BND_REPLICATE) {  // see tile_step_replicate_border
        const int x1 = c.gx + 32;
        c.jc0 = c.j + (min(max(c.gx, 0), w - 1) - c.gx);
        c.jc1 = c.j + 32 + (min(max(x1, 0), w - 1) - x1);
        c.st0 = (c.gx >= -1) & (c.gx <= w);
        c.st1 = (x1 >= -1) & (x1 <= w);
    } else {
        c.jc0 = c.j;
        c.jc1 = c.j + 32;
        c.st0 = c.cin0;
        c.st1 = c.cin1;
    }
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
        // f at the columns the cells are computed at (REPLICATE: a ring-column cell takes its
        // source cell's f)
        const S *fr = jb.f + (int64_t)(Y0 + c.ib) * jb.ld + X0;
        const bool hasf = jb.f != nullptr;
#pragma unroll
        for (int k = 0; k < kRY; ++k) {
            // predicated loads, no branch
            const bool rk = hasf & ((in_rows >> k) & 1u);
            const S *fk = fr + (int64_t)k * jb.ld;
            const float a = (rk & c.st0) ? Store<S>::load(fk + c.jc0) : 0.0f;
            const float b = (rk & c.st1) ? Store<S>::load(fk + c.jc1) : 0.0f;
            g[k] = __fmul2_rn(cf, make_float2(a, b));
        }
    }

    // ---- wait for the window: thread 0 waits on the barrier (its completion makes the copied
    // data visible to it), then the CTA barrier orders everyone else's reads after that
    if (jb.use_tma) {
        const bool ok = (tid != 0) || mbar_wait_bounded(smem_u32(bar), phase, kWaitLimitNs);
        if (__syncthreads_or(!ok)) {
            if (tid == 0) {
                if (status) atomicOr(status, 1u);
                // the copies may still land: wait for them (bounded) before the CTA's shared
                // memory is released
                mbar_wait_bounded(smem_u32(bar), phase, kWaitLimitNs);
            }
            return false;
        }
        if (ftma) {  // f as loaded by TMA: zero outside the image, like the plain loads' predicates
            const S *fr = static_cast<const S *>(fwin) + c.ib * LW;
#pragma unroll
            for (int k = 0; k < kRY; ++k)
                g[k] = __fmul2_rn(cf, make_float2(Store<S>::to_float(fr[k * LW + c.jc0]),
                                                  Store<S>::to_float(fr[k * LW + c.jc1])));
        }
        if constexpr (sizeof(S) != 4) {  // widen the staged 16-bit box, 8 elements per 16-byte access
            static_assert((LH * LW) % 8 == 0, "the staged box is a whole number of 16-byte chunks");
            const uint4 *st4 = static_cast<const uint4 *>(stage);
            float4 *dst4 = reinterpret_cast<float4 *>(buf0);
            for (int q = tid; q < LH * LW / 8; q += NT) {
                const uint4 raw = st4[q];
                const float2 a = Store<S>::unpack2(raw.x), b = Store<S>::unpack2(raw.y);
                const float2 c2 = Store<S>::unpack2(raw.z), d2 = Store<S>::unpack2(raw.w);
                dst4[2 * q] = make_float4(a.x, a.y, b.x, b.y);
                dst4[2 * q + 1] = make_float4(c2.x, c2.y, d2.x, d2.y);
            }
            // the widened window is complete, and every thread has read f from buffer 1
            __syncthreads();
        }
    } else {
        __syncthreads();
    }

    // ---- REPLICATE: fill the ring just outside the image from its nearest in-image cell.
    if (BND == BND_REPLICATE && border) {
        refresh_ring<S, LH, NT>(buf0, X0, Y0, h, w, tid);
        __syncthreads();
    }

    // ---- T steps: ping-pong buf0 -> buf1 -> buf0 ...; the last one writes the output tile.
    // A warp whose cells all lie beyond the ring just outside the image (rows >= h + 1, or
    // columns >= w + 1: tiles that overhang the image's bottom or right edge) has nothing that
    // any in-image cell reads, so it skips the arithmetic (it still takes part in the barriers).
    const int lane0 = c.gx - lane;
    const bool idle = (Y0 + c.ib >= h + 1) | (lane0 >= w + 1);
    auto one_step = [&](int s) {
        const float *src = (s & 1) ? buf1 : buf0;
        float *dst = (s & 1) ? buf0 : buf1;
        if (!border) {
            tile_step<WRITE_INTERIOR, S, BND, NW>(src, dst, c, g);
            __syncthreads();
        } else {
            if (!idle) {
                if constexpr (BND == BND_REPLICATE)
                    tile_step_replicate_border<S, NW>(src, dst, c, g);
                else
                    tile_step<WRITE_BORDER, S, BND, NW>(src, dst, c, g);
            }
            __syncthreads();
        }
    };
    // Single images and 16-warp batch tiles unroll the T - 1 steps (T is a template parameter):
    // 2.3 % faster at 4096^2 than a loop, whose pointer selection and back edge each step paid;
    // the 512-image batch 643.5 -> 648.0 Gpix-iter/s.  8-warp batch tiles keep the loop: unrolled
    // they ran slower at T >= 4.
    if constexpr (UNROLL) {
#pragma unroll
        for (int s = 0; s < T - 1; ++s) one_step(s);
    } else {
#pragma unroll 1
        for (int s = 0; s < T - 1; ++s) one_step(s);
    }
    if (idle) return true;  // none of its cells is an output cell inside the image
    int64_t ldo;
    S *out = out_of(&ldo);
    tile_step<WRITE_GLOBAL, S, BND, NW>(((T - 1) & 1) ? buf1 : buf0, nullptr, c, g,
                                        out + (int64_t)(Y0 + c.ib) * ldo + c.gx, ldo);
    return true;
}

// Thread 0 of a tile of a chained launch: wait (bounded) until the 3 x 3 tiles around (tx, ty) of
// the previous launch have stored a flag >= need.  Their outputs are this window's U^t (a window
// reaches at most T + 4 < one tile into its neighbours), and they are the only tiles of that
// launch whose windows cover this tile's output region, so their completion also ends every read
// of it.  Every tile they wait for is already running: a chained launch is scheduled only once
// every CTA of the previous one has started.  A wait that gives up sets bit 0 of the status word
// (and then the load goes ahead: the run's result is reported as failed); a tile that finds the
// bit set does not wait, so one late tile does not make every later one wait out its limit.
__device__ __forceinline__ void wait_tile_flags(const unsigned int *flags, int tx, int ty, int ntx, int nty,
                                                unsigned int need, unsigned int *status) {
    // the least of the nine flags, read at once (relaxed loads: one memory round trip); only a
    // tile whose neighbours are not all done polls again
    auto least = [&]() {
        unsigned int v[9];
#pragma unroll
        for (int q = 0; q < 9; ++q) {  // all nine loads issued before any result is used
            const int x = tx + q % 3 - 1, y = ty + q / 3 - 1;
            v[q] = ((x >= 0) & (x < ntx) & (y >= 0) & (y < nty)) ? ld_relaxed_gpu(flags + (int64_t)y * ntx + x)
                                                                 : need;
        }
        unsigned int low = need;
#pragma unroll
        for (int q = 0; q < 9; ++q) low = min(low, v[q]);
        return low;
    };
    if (least() < need) {
        const uint64_t t0 = global_timer_ns();
        for (;;) {
            __nanosleep(64);
            if (least() >= need) break;
            if (status && (*static_cast<volatile unsigned int *>(status) & 1u)) break;  // another wait gave up
            if (global_timer_ns() - t0 > kWaitLimitNs) {
                if (status) atomicOr(status, 1u);
                break;
            }
        }
    }
    // the relaxed loads that saw the flags, then this fence: an acquire of the neighbours' release
    // stores; then what it made visible is ordered before this thread's TMA reads
    __threadfence();
    fence_proxy_async_global();
}

template <int T, typename S, int BND, bool BATCH, int NW>
__global__ void __launch_bounds__(32 * NW, 32 / NW)
    tile_flow_kernel(const __grid_constant__ CUtensorMap tmap, const __grid_constant__ CUtensorMap fmap,
                     const TileParams p) {
    using G = TGeom<S, NW>;
    extern __shared__ unsigned char smem_raw[];
    __shared__ __align__(8) uint64_t bar;
    // 128-byte aligned start of the buffers, formed as an offset into the __shared__ array (not
    // through an integer cast) so that every access below stays a shared-memory access
    float *buf0 = reinterpret_cast<float *>(smem_raw + ((128u - (smem_u32(smem_raw) & 127u)) & 127u));
    float *buf1 = buf0 + G::BUF;

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
    // U^t ready: the tiles of the previous launch that this one depends on (flags), else that
    // whole launch
    auto wait_input = [&](bool late) {
        const bool by_flags = !BATCH && p.flag_wait > 0;
        if (by_flags && !late) {
            const int ty = blockIdx.x / p.ntx, tx = blockIdx.x - ty * p.ntx;
            wait_tile_flags(p.flags, tx, ty, p.ntx, ((int)gridDim.x) / p.ntx, (unsigned)p.flag_wait, p.status);
        } else if (!by_flags && late) {
            griddep_wait();
        }
    };
    // the next launch may be scheduled once every CTA of this one is running
    griddep_launch_dependents();
    if (jb.use_tma && threadIdx.x == 0) mbar_init(smem_u32(&bar), 1);
    // the output pointer is looked up again after the steps (kernel parameters, or the image
    // descriptor in L1) rather than kept in registers through them
    tile_job<T, S, BND, NW, !BATCH || NW == 16>(jb, p.owt, p.oht, p.status, buf0, buf1, &bar, 0u, [&](int64_t *ldo) -> S * {
        if (BATCH) {
            const BatchImage &im = p.images[p.tiles[blockIdx.x].x];
            *ldo = p.dst_role == 1 ? im.ld_out : im.ld;
            return static_cast<S *>(const_cast<void *>(im.buf[p.dst_role]));
        }
        *ldo = p.ld_out;
        return static_cast<S *>(p.out);
    }, wait_input);
    // publish this tile's completion: every thread's output stores (and its reads of U^t) come
    // before the CTA barrier, and so before thread 0's release store of the flag
    if (!BATCH && p.flag_set > 0) {
        __syncthreads();
        if (threadIdx.x == 0) st_release_gpu(p.flags + blockIdx.x, (unsigned)p.flag_set);
    }
}

template <int T, typename S, int BND, bool BATCH, int NW>
cudaError_t launch_tile_t(const CUtensorMap *map, TileParams p, int64_t nblocks, cudaStream_t st) {
    using G = TGeom<S, NW>;
    if (!BATCH) {
        p.owt = kCW + 2 - 2 * T;
        p.oht = G::CH + 2 - 2 * T;
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
        e = cudaFuncSetAttribute(tile_flow_kernel<T, S, BND, BATCH, NW>,
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
        tile_flow_kernel<T, S, BND, BATCH, NW><<<(unsigned)nblocks, G::THREADS, G::SMEM, st>>>(map[0], map[1], p);
        return cudaGetLastError();
    }
    cudaLaunchConfig_t cfg{};
    cfg.gridDim = dim3((unsigned)nblocks);
    cfg.blockDim = dim3(G::THREADS);
    cfg.dynamicSmemBytes = G::SMEM;
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, tile_flow_kernel<T, S, BND, BATCH, NW>, map[0], map[1], p);
}

// steps = T (1..8), tile = 1 or 2 (tile_warps); batch_tiles >= 0: a batch launch over that many
// tiles of the plan's table, < 0: a single-image launch
template <typename S, int BND, int NW>
cudaError_t launch_tile_steps_nw(int steps, const CUtensorMap *map, const TileParams &p,
                                 int64_t batch_tiles, cudaStream_t st) {
    const bool b = batch_tiles >= 0;
#define WMC_TILE_CASE(T)                                                                        \
    case T:                                                                                     \
        return b ? launch_tile_t<T, S, BND, true, NW>(map, p, batch_tiles, st)                  \
                 : launch_tile_t<T, S, BND, false, NW>(map, p, 0, st);
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
