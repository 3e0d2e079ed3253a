// wmc_tile.cuh -- temporally blocked WMC stencil kernel (eval and Jacobi flow steps).
//
// One CTA owns an output tile and takes T Jacobi steps of
//     U^{t+1} = U^t + step (lambda H^w(U^t) - mu (U^t - f))     (Sec. V-B, Eq. MCF)
// entirely in shared memory before writing the tile back.  This is exact because the update
// is Jacobi-ordered: every pixel of step t+1 reads only U^t, so after T steps a cell is
// correct if the (2T+1)^2 cells around it were loaded.  The CTA loads a (CW+2) x (CH+2)
// window (ring of T cells around the (CW+2-2T) x (CH+2-2T) output tile), updates the inner
// CW x CH cells each step, and its error front moves in one cell per step.
//
// Image boundary.  REPLICATE: neighbour reads of in-image cells are clamped to the image
// (row and column indices), so cells outside the image are never read after the load and
// are never written.  ZERO: cells outside the image hold 0 in both buffers and are never
// written, and reads are not clamped.
//
// Thread layout: 8 warps; warp g owns rows 1+8g .. 8+8g of the update region, lane l owns
// columns 1+l and 33+l.  Each thread reads its column triple (c-1, c, c+1) for its 8 rows plus
// one row above and below (30 conflict-free shared loads per column per step: every warp
// instruction reads 32 consecutive words of one row) and keeps f * step * mu for its 16
// cells in registers for the whole launch.
#pragma once

#include "wmc_device.cuh"
#include "wmc_internal.h"

namespace wmc {

constexpr int SW = kTileCW + 2;  // shared tile width
constexpr int SH = kTileCH + 2;  // shared tile height
constexpr int SP = SW;           // shared pitch (warp reads are row-contiguous: no conflicts)
constexpr int RY = kTileCH / 8;  // rows per warp
constexpr int NCOL = kTileCW / 32;

template <int T, int MODE, typename S, int BND>
__global__ void __launch_bounds__(kTileThreads, 2) tile_kernel(const TileParams p) {
    extern __shared__ float smem[];

    constexpr int OW = SW - 2 * T;
    constexpr int OH = SH - 2 * T;
    const int h = p.h, w = p.w;
    const int x0 = blockIdx.x * OW;  // first output column of this CTA
    const int y0 = blockIdx.y * OH;
    const int gx0 = x0 - T;          // image column of shared column 0
    const int gy0 = y0 - T;
    const S *__restrict__ u = static_cast<const S *>(p.u);

    // ---- load the (SH x SW) window of U^t
    for (int i = threadIdx.x; i < SH * SW; i += kTileThreads) {
        const int r = i / SW, c = i - (i / SW) * SW;
        int gy = gy0 + r, gx = gx0 + c;
        const bool in = (gy >= 0) & (gy < h) & (gx >= 0) & (gx < w);
        float v;
        if (BND == BND_ZERO) {
            v = in ? Store<S>::load(u + (int64_t)gy * p.ldu + gx) : 0.0f;
        } else {
            gy = min(max(gy, 0), h - 1);
            gx = min(max(gx, 0), w - 1);
            v = Store<S>::load(u + (int64_t)gy * p.ldu + gx);
        }
        smem[r * SP + c] = v;
        if (T > 1) smem[SH * SP + r * SP + c] = v;
    }

    const int lane = threadIdx.x & 31;
    const int warp = threadIdx.x >> 5;
    const int rbeg = 1 + warp * RY;  // first shared row this thread updates

    // Image extent in shared coordinates (for clamping and for the in-image test).
    const int rTop = -gy0, rBot = h - 1 - gy0;
    const int cLft = -gx0, cRgt = w - 1 - gx0;

    // Clamped shared row offsets of rows rbeg-1 .. rbeg+RY (fixed for the whole launch).
    int roff[RY + 2];
#pragma unroll
    for (int k = 0; k < RY + 2; ++k) {
        int r = rbeg - 1 + k;
        if (BND == BND_REPLICATE) r = min(max(r, rTop), rBot);
        roff[k] = r * SP;
    }
    int cc[NCOL], cl[NCOL], cr[NCOL];
#pragma unroll
    for (int j = 0; j < NCOL; ++j) {
        cc[j] = 1 + lane + 32 * j;
        cl[j] = cc[j] - 1;
        cr[j] = cc[j] + 1;
        if (BND == BND_REPLICATE) {
            cl[j] = max(cl[j], cLft);
            cr[j] = min(cr[j], cRgt);
        }
    }

    // step*mu*f for the 16 owned cells (0 outside the image or for the pure flow).
    float g[NCOL][RY];
    const bool use_f = (MODE == MODE_FLOW) && (p.f != nullptr);
#pragma unroll
    for (int j = 0; j < NCOL; ++j)
#pragma unroll
        for (int k = 0; k < RY; ++k) {
            const int gy = gy0 + rbeg + k, gx = gx0 + cc[j];
            float fv = 0.0f;
            if (use_f && gy >= 0 && gy < h && gx >= 0 && gx < w)
                fv = Store<S>::load(static_cast<const S *>(p.f) + (int64_t)gy * p.ldf + gx);
            g[j][k] = p.c_f * fv;
        }
    __syncthreads();

    S *__restrict__ out = static_cast<S *>(p.out);

#pragma unroll 1
    for (int s = 0; s < T; ++s) {
        const float *src = smem + (s & 1) * (SH * SP);
        float *dst = smem + ((s + 1) & 1) * (SH * SP);
        const bool last = (s == T - 1);
#pragma unroll
        for (int j = 0; j < NCOL; ++j) {
            // Sliding 3-row window over columns c-1 (a), c (b), c+1 (d).
            float a0 = src[roff[0] + cl[j]], b0 = src[roff[0] + cc[j]], d0 = src[roff[0] + cr[j]];
            float a1 = src[roff[1] + cl[j]], b1 = src[roff[1] + cc[j]], d1 = src[roff[1] + cr[j]];
            const int gx = gx0 + cc[j];
            const bool col_in = (gx >= 0) & (gx < w);
#pragma unroll
            for (int k = 0; k < RY; ++k) {
                const float a2 = src[roff[k + 2] + cl[j]];
                const float b2 = src[roff[k + 2] + cc[j]];
                const float d2 = src[roff[k + 2] + cr[j]];
                const float h12 = half_laplace12(a0, b0, d0, a1, b1, d1, a2, b2, d2);
                const int r = rbeg + k;
                const int gy = gy0 + r;
                const bool in = col_in & (gy >= 0) & (gy < h);
                float v;
                if (MODE == MODE_EVAL) {
                    v = p.c_h * h12;
                } else {
                    v = fmaf(p.c_h, h12, fmaf(p.c_keep, b1, g[j][k]));
                }
                if (!last) {
                    if (in) dst[r * SP + cc[j]] = Store<S>::round(v);
                } else {
                    // Output cells: shared rows/cols T .. T+OH-1 / T .. T+OW-1.
                    const bool own = (r >= T) & (r < T + OH) & (cc[j] >= T) & (cc[j] < T + OW);
                    if (in & own) Store<S>::store(out + (int64_t)gy * p.ldo + gx, v);
                }
                a0 = a1; b0 = b1; d0 = d1;
                a1 = a2; b1 = b2; d1 = d2;
            }
        }
        if (!last) __syncthreads();
    }
    (void)rTop; (void)rBot; (void)cLft; (void)cRgt;
}

template <int T, int MODE, typename S, int BND>
cudaError_t launch_tile_t(const TileParams &p, cudaStream_t st) {
    constexpr int OW = SW - 2 * T;
    constexpr int OH = SH - 2 * T;
    dim3 grid((p.w + OW - 1) / OW, (p.h + OH - 1) / OH);
    const size_t smem = (T > 1 ? 2 : 1) * SH * SP * sizeof(float);
    tile_kernel<T, MODE, S, BND><<<grid, kTileThreads, smem, st>>>(p);
    return cudaGetLastError();
}

template <typename S, int BND>
cudaError_t launch_tile_steps(int mode, int steps, const TileParams &p, cudaStream_t st) {
    if (mode == MODE_EVAL) return launch_tile_t<1, MODE_EVAL, S, BND>(p, st);
    switch (steps) {
        case 1: return launch_tile_t<1, MODE_FLOW, S, BND>(p, st);
        case 2: return launch_tile_t<2, MODE_FLOW, S, BND>(p, st);
        case 3: return launch_tile_t<3, MODE_FLOW, S, BND>(p, st);
        case 4: return launch_tile_t<4, MODE_FLOW, S, BND>(p, st);
        case 5: return launch_tile_t<5, MODE_FLOW, S, BND>(p, st);
        case 6: return launch_tile_t<6, MODE_FLOW, S, BND>(p, st);
        case 7: return launch_tile_t<7, MODE_FLOW, S, BND>(p, st);
        case 8: return launch_tile_t<8, MODE_FLOW, S, BND>(p, st);
        default: return cudaErrorInvalidValue;
    }
}

template <typename S>
cudaError_t launch_tile_dtype(int mode, int steps, const TileParams &p, cudaStream_t st) {
    if (p.bnd == BND_ZERO) return launch_tile_steps<S, BND_ZERO>(mode, steps, p, st);
    return launch_tile_steps<S, BND_REPLICATE>(mode, steps, p, st);
}

}  // namespace wmc
