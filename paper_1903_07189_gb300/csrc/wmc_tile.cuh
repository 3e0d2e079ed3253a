// wmc_tile.cuh -- temporally blocked WMC flow kernel: T >= 2 Jacobi steps per launch in shared
// memory.
//
// The update U^{t+1} = U^t + step (lambda H^w(U^t) - mu (U^t - f)) (Sec. V-B, Eq. MCF) is
// Jacobi-ordered: every pixel of step t+1 reads only U^t.  So a CTA can load a window of U^t,
// take T steps on it without talking to anyone, and write back the part of the window that is
// still exact: each step's stale border moves one cell inwards.
//
// Geometry (element coordinates; X0, Y0 = global position of shared cell (0,0)):
//   loaded window  [X0, X0+LW) x [Y0, Y0+LH)       one 2-D TMA box, zero-filled outside the image
//   updated cells  [X0+2, X0+2+CW) x [Y0+1, Y0+1+CH)    every step (CW = 128, CH = 64)
//   exact after T  [X0+1+T, X0+3+CW-T) x [Y0+T, Y0+2+CH-T)
//   written back   [x0, x0+OW) x [y0, y0+OH),  x0 = X0 + M, y0 = Y0 + T
// M (>= T+1) and OW are multiples of the TMA alignment (16 bytes of elements), so every TMA
// x-coordinate is aligned and every thread's column pair (even, odd) is either wholly inside or
// wholly outside the output tile.
//
// Threads: 16 warps as 2 (x) x 8 (y); lane l of warp (wx, wy) updates columns j = 2 + 64 wx + l
// and j + 32 for rows i = 1 + 8 wy .. 8 + 8 wy.  The two columns are the two lanes of packed
// FP32x2 arithmetic: every operand pair (west, centre, east neighbours of both cells) is read
// by two conflict-free 4-byte shared loads straight into an aligned register pair, so no
// register shuffling is needed (pairing the adjacent columns j, j+1 instead would make six of
// the nine operands straddle register pairs).  Offsets are constants: the inner loop has no index
// arithmetic and no per-cell predicates in tiles that lie inside the image.
//
// Image boundary.  ZERO: the TMA fill supplies the zeros; in tiles touching the border, cells
// outside the image are rewritten as 0 every step.  REPLICATE: the ring of cells just outside
// the image is kept equal to its nearest in-image cell (filled after the load, then rewritten
// by the in-image edge cells every step), so in-image cells read their neighbours without any
// clamping and produce exactly what clamped reads would.
//
// Shared memory always holds FP32; for BF16/FP16 storage the TMA box lands in a staging area
// and is widened once, and every step rounds its result to the storage type, so the arithmetic
// is identical to the single-step streaming kernel.
#pragma once

#include <cuda.h>
#include <string.h>

#include "wmc_device.cuh"
#include "wmc_internal.h"

namespace wmc {

constexpr int kCW = 128;   // updated columns per step
constexpr int kCH = 64;    // updated rows per step
constexpr int kRY = 8;     // rows per thread
constexpr int kTileWX = 2; // warps across (64 columns each)
constexpr int kTileWY = kCH / kRY;  // warps down
constexpr int kTileThreadsV2 = 32 * kTileWX * kTileWY;  // 512

template <typename S> struct Geom {
    static constexpr int A = 16 / (int)sizeof(S);                 // TMA x alignment (elements)
    static constexpr int LW = ((kCW + 3 + A - 1) / A) * A;        // loaded width
    static constexpr int LH = kCH + 2;                            // loaded height
    static constexpr int P = LW;                                  // shared pitch (floats)
    static constexpr int BUF = LH * P;                            // floats per buffer
    static constexpr int STAGE_BYTES = sizeof(S) == 4 ? 0 : LH * LW * (int)sizeof(S);
    static constexpr int SMEM = 2 * BUF * 4 + STAGE_BYTES + 128;  // + alignment slack
};

// Output tile of a T-step launch: margin M (>= T+1, TMA-aligned), width OW, height OH.
template <typename S, int T> struct Out {
    static constexpr int A = Geom<S>::A;
    static constexpr int M = A * ((T + 1 + A - 1) / A);
    static constexpr int OW = A * ((kCW + 3 - T - M) / A);
    static constexpr int OH = kCH + 2 - 2 * T;
};

struct TileV2Params {
    const void *u;    // U^t (device); read through the tensor map when use_tma
    const void *f;    // f or nullptr (mean-curvature flow)
    void *out;        // U^{t+T}
    int64_t ldu, ldf, ldo;
    int32_t h, w;
    int32_t ntx;      // tiles per row of tiles
    int32_t use_tma;
    int32_t vec_f;    // f rows allow 2-element loads (aligned base, even pitch)
    int32_t vec_o;    // same for the output
    float c_keep, c_f, c_h;
    unsigned int *status;  // device status word (bit 0: a bounded wait gave up) or nullptr
};

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

__device__ __forceinline__ void tma_load_2d(uint32_t dst, const CUtensorMap *map, int x, int y,
                                            uint32_t bar) {
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.tile.mbarrier::complete_tx::bytes"
        " [%0], [%1, {%2, %3}], [%4];" ::"r"(dst),
        "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(bar)
        : "memory");
}

// Poll the barrier's phase; give up after `limit_ns` (returns false).
__device__ __forceinline__ bool mbar_wait_bounded(uint32_t bar, uint32_t phase, uint64_t limit_ns) {
    const uint64_t t0 = global_timer_ns();
    for (;;) {
        uint32_t done;
        asm volatile(
            "{ .reg .pred p; mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;"
            " selp.u32 %0, 1, 0, p; }"
            : "=r"(done)
            : "r"(bar), "r"(phase)
            : "memory");
        if (done) return true;
        if (global_timer_ns() - t0 > limit_ns) return false;
    }
}

constexpr uint64_t kWaitLimitNs = 200ull * 1000 * 1000;  // 0.2 s

__device__ __forceinline__ float2 lds2(const float *p) {
    return *reinterpret_cast<const float2 *>(p);
}
__device__ __forceinline__ void sts2(float *p, float a, float b) {
    *reinterpret_cast<float2 *>(p) = make_float2(a, b);
}

// ------------------------------------------------------------------------------- kernel
// Per-thread constants of one tile.
struct TileCtx {
    int j, ib;         // shared column of the thread's first cell (second: j + 32), first row
    int X0, Y0, gx;    // window origin, image column of the first cell
    int h, w;
    bool cin0, cin1;   // the two cells' columns lie inside the image
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
template <int WMODE, int T, typename S, int BND>
__device__ __forceinline__ void tile_step(const float *__restrict__ src, float *__restrict__ dst,
                                          const TileCtx &c, const float2 (&g)[kRY],
                                          const TileV2Params &p) {
    using G = Geom<S>;
    constexpr int P = G::P, LH = G::LH, LW = G::LW;
    constexpr int M = Out<S, T>::M, OW = Out<S, T>::OW, OH = Out<S, T>::OH;
    const float2 ch = make_float2(p.c_h, p.c_h), ck = make_float2(p.c_keep, p.c_keep);
    const float *rp = src + (c.ib - 1) * P + c.j;
    Row3 r0 = load_row3(rp), r1 = load_row3(rp + P);
    const bool col_out0 = (c.j >= M) & (c.j < M + OW);
    const bool col_out1 = (c.j + 32 >= M) & (c.j + 32 < M + OW);
#pragma unroll
    for (int k = 0; k < kRY; ++k) {
        const Row3 r2 = load_row3(rp + (k + 2) * P);
        const float2 hw = half_laplace12_x2(r0.w, r0.c, r0.e, r1.w, r1.c, r1.e, r2.w, r2.c, r2.e);
        float2 v = __ffma2_rn(ch, hw, __ffma2_rn(ck, r1.c, g[k]));
        const int i = c.ib + k;
        if (WMODE == WRITE_INTERIOR) {
            float *d = dst + i * P + c.j;
            d[0] = Store<S>::round(v.x);
            d[32] = Store<S>::round(v.y);
        } else if (WMODE == WRITE_BORDER) {
            v.x = Store<S>::round(v.x);
            v.y = Store<S>::round(v.y);
            const int gy = c.Y0 + i;
            const bool rin = (gy >= 0) & (gy < c.h);
#pragma unroll
            for (int e = 0; e < 2; ++e) {
                const bool in = rin & (e == 0 ? c.cin0 : c.cin1);
                const float ve = e == 0 ? v.x : v.y;
                const int jc = c.j + 32 * e;
                if (BND == BND_ZERO) {
                    dst[i * P + jc] = in ? ve : 0.0f;
                } else {
                    // in-image cells: normal write; cells on the image edge also refresh the
                    // ring cells outside the image that copy them
                    if (!in) continue;
                    const int xe = c.gx + 32 * e;
                    dst[i * P + jc] = ve;
                    if ((gy == 0) | (gy == c.h - 1) | (xe == 0) | (xe == c.w - 1)) {
                        const int up = (gy == 0) ? -1 : 0, dn = (gy == c.h - 1) ? 1 : 0;
                        const int lf = (xe == 0) ? -1 : 0, rt = (xe == c.w - 1) ? 1 : 0;
                        for (int di = up; di <= dn; ++di)
                            for (int dj = lf; dj <= rt; ++dj) {
                                if (di == 0 && dj == 0) continue;
                                const int ii = i + di, jj = jc + dj;
                                if (ii >= 0 && ii < LH && jj >= 0 && jj < LW) dst[ii * P + jj] = ve;
                            }
                    }
                }
            }
        } else {
            const int gy = c.Y0 + i;
            if ((i >= T) & (i < T + OH) & (gy < c.h)) {
                S *o = static_cast<S *>(p.out) + (int64_t)gy * p.ldo + c.gx;
                if (col_out0 & (c.gx < c.w)) Store<S>::store(o, v.x);
                if (col_out1 & (c.gx + 32 < c.w)) Store<S>::store(o + 32, v.y);
            }
        }
        r0 = r1;
        r1 = r2;
    }
}

template <int T, typename S, int BND>
__global__ void __launch_bounds__(kTileThreadsV2, 2)
    tile_v2_kernel(const __grid_constant__ CUtensorMap tmap, const TileV2Params p) {
    using G = Geom<S>;
    constexpr int LW = G::LW, LH = G::LH, P = G::P, BUF = G::BUF;
    constexpr int M = Out<S, T>::M;
    constexpr int OW = Out<S, T>::OW;
    constexpr int OH = Out<S, T>::OH;
    static_assert(OW > 0 && OH > 0, "tile too small for T");

    extern __shared__ unsigned char smem_raw[];
    __shared__ __align__(8) uint64_t bar;
    float *buf0 = reinterpret_cast<float *>(
        (reinterpret_cast<uintptr_t>(smem_raw) + 127) & ~uintptr_t(127));
    float *buf1 = buf0 + BUF;

    const int h = p.h, w = p.w;
    const int ty = blockIdx.x / p.ntx, tx = blockIdx.x - ty * p.ntx;
    const int x0 = tx * OW, y0 = ty * OH;
    const int X0 = x0 - M, Y0 = y0 - T;
    const int tid = threadIdx.x;
    const bool border = (X0 < 0) | (Y0 < 0) | (X0 + LW > w) | (Y0 + LH > h);

    // ---- issue the load of the window of U^t
    if (p.use_tma) {
        if (tid == 0) mbar_init(smem_u32(&bar), 1);
        __syncthreads();
        if (tid == 0) {
            void *dst = (sizeof(S) == 4) ? static_cast<void *>(buf0)
                                         : static_cast<void *>(buf1 + BUF);  // staging
            mbar_expect_tx(smem_u32(&bar), (uint32_t)(LW * LH * sizeof(S)));
            tma_load_2d(smem_u32(dst), &tmap, X0, Y0, smem_u32(&bar));
        }
    } else {
        const S *u = static_cast<const S *>(p.u);
        for (int idx = tid; idx < LH * LW; idx += kTileThreadsV2) {
            const int i = idx / LW, j = idx - (idx / LW) * LW;
            const int gy = Y0 + i, gx = X0 + j;
            float v = 0.0f;
            if (gy >= 0 && gy < h && gx >= 0 && gx < w) v = Store<S>::load(u + (int64_t)gy * p.ldu + gx);
            buf0[i * P + j] = v;
        }
    }

    // ---- per-thread geometry and f (overlaps the load)
    const int lane = tid & 31, warp = tid >> 5;
    TileCtx c;
    c.j = 2 + 64 * (warp & 1) + lane;
    c.ib = 1 + kRY * (warp >> 1);
    c.X0 = X0;
    c.Y0 = Y0;
    c.gx = X0 + c.j;
    c.h = h;
    c.w = w;
    c.cin0 = (c.gx >= 0) & (c.gx < w);
    c.cin1 = (c.gx + 32 >= 0) & (c.gx + 32 < w);
    float2 g[kRY];
    {
        const S *f = static_cast<const S *>(p.f);
        const int gx = c.gx;
#pragma unroll
        for (int k = 0; k < kRY; ++k) {
            const int gy = Y0 + c.ib + k;
            float a = 0.0f, b = 0.0f;
            if (f != nullptr && gy >= 0 && gy < h) {
                const S *fr = f + (int64_t)gy * p.ldf;
                if (c.cin0) a = Store<S>::load(fr + gx);
                if (c.cin1) b = Store<S>::load(fr + gx + 32);
            }
            g[k] = __fmul2_rn(make_float2(p.c_f, p.c_f), make_float2(a, b));
        }
    }

    // ---- wait for the window
    if (p.use_tma) {
        const bool ok = mbar_wait_bounded(smem_u32(&bar), 0, kWaitLimitNs);
        if (__syncthreads_or(!ok)) {
            if (tid == 0 && p.status) atomicOr(p.status, 1u);
            return;
        }
        if (sizeof(S) != 4) {  // widen the staged 16-bit box
            const S *stage = reinterpret_cast<const S *>(buf1 + BUF);
            for (int idx = tid; idx < LH * LW; idx += kTileThreadsV2)
                buf0[idx] = Store<S>::to_float(stage[idx]);
            __syncthreads();
        }
    } else {
        __syncthreads();
    }

    // ---- REPLICATE: fill the ring just outside the image from its nearest in-image cell.
    // The ring is at most four segments (image rows -1 and h, image columns -1 and w) crossing
    // the window; corner cells belong to two segments and get the same value from both.
    if (BND == BND_REPLICATE && border) {
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
                const int u = t - 2 * LW;
                j2 = (u < LH) ? jc0 : jc1;
                i = (u < LH) ? u : u - LH;
                if (j2 < 0 || j2 >= LW || i < ilo || i > ihi) continue;
            }
            const int yy = Y0 + i, xx = X0 + j2;
            const int ci = min(max(yy, 0), h - 1) - Y0, cj = min(max(xx, 0), w - 1) - X0;
            buf0[i * P + j2] = buf0[ci * P + cj];
        }
        __syncthreads();
    }

    // ---- T steps: ping-pong buf0 -> buf1 -> buf0 ...; the last one writes the output tile
#pragma unroll 1
    for (int s = 0; s < T - 1; ++s) {
        const float *src = (s & 1) ? buf1 : buf0;
        float *dst = (s & 1) ? buf0 : buf1;
        if (!border)
            tile_step<WRITE_INTERIOR, T, S, BND>(src, dst, c, g, p);
        else
            tile_step<WRITE_BORDER, T, S, BND>(src, dst, c, g, p);
        __syncthreads();
    }
    tile_step<WRITE_GLOBAL, T, S, BND>(((T - 1) & 1) ? buf1 : buf0, nullptr, c, g, p);
}

template <int T, typename S, int BND>
cudaError_t launch_tile_v2_t(const CUtensorMap *map, TileV2Params p, cudaStream_t st) {
    using G = Geom<S>;
    constexpr int OW = Out<S, T>::OW;
    constexpr int OH = Out<S, T>::OH;
    const int64_t ntx = (p.w + OW - 1) / OW, nty = (p.h + OH - 1) / OH;
    if (ntx * nty > 0x7fffffffLL) return cudaErrorInvalidConfiguration;
    p.ntx = (int32_t)ntx;
    cudaError_t e = cudaFuncSetAttribute(tile_v2_kernel<T, S, BND>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, G::SMEM);
    if (e != cudaSuccess) return e;
    CUtensorMap dummy;
    if (!p.use_tma) {
        memset(&dummy, 0, sizeof dummy);
        map = &dummy;
    }
    tile_v2_kernel<T, S, BND><<<(unsigned)(ntx * nty), kTileThreadsV2, G::SMEM, st>>>(*map, p);
    return cudaGetLastError();
}

template <typename S, int BND>
cudaError_t launch_tile_v2_steps(int steps, const CUtensorMap *map, const TileV2Params &p,
                                 cudaStream_t st) {
    switch (steps) {
        case 2: return launch_tile_v2_t<2, S, BND>(map, p, st);
        case 3: return launch_tile_v2_t<3, S, BND>(map, p, st);
        case 4: return launch_tile_v2_t<4, S, BND>(map, p, st);
        case 5: return launch_tile_v2_t<5, S, BND>(map, p, st);
        case 6: return launch_tile_v2_t<6, S, BND>(map, p, st);
        case 7: return launch_tile_v2_t<7, S, BND>(map, p, st);
        case 8: return launch_tile_v2_t<8, S, BND>(map, p, st);
        default: return cudaErrorInvalidValue;
    }
}

template <typename S>
cudaError_t launch_tile_v2_dtype(int steps, int bnd, const CUtensorMap *map,
                                 const TileV2Params &p, cudaStream_t st) {
    if (bnd == BND_ZERO) return launch_tile_v2_steps<S, BND_ZERO>(steps, map, p, st);
    return launch_tile_v2_steps<S, BND_REPLICATE>(steps, map, p, st);
}

}  // namespace wmc
