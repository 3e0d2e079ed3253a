// wmc_stream.cuh -- single-pass WMC kernels (one evaluation, or one Jacobi step) that stream the
// image through registers.  These passes read each input pixel once and are bound by HBM
// bandwidth, so the kernel is built to keep many loads in flight and spend few instructions per
// pixel:
//   - a warp owns 64 consecutive columns, each lane a pair (x, x+1) loaded as one 8-byte (FP32)
//     or 4-byte (16-bit) access; the left/right neighbour columns come from the adjacent lanes by
//     warp shuffle, and only lanes 0 and 31 load one extra column each;
//   - a thread walks down a strip of RY rows, keeping a 3-row window in registers, so every row
//     is loaded once per thread (the rows above and below the strip are re-read by the
//     neighbouring strip, from L2);
//   - the boundary rule is applied while loading (REPLICATE: clamped index; ZERO: 0 outside),
//     so the arithmetic never branches on position.
#pragma once

#include "wmc_device.cuh"
#include "wmc_internal.h"

namespace wmc {

constexpr int kStreamWarps = 8;
constexpr int kStreamRY = 8;

struct StreamParams {
    const void *u;
    const void *f;  // flow only; nullptr = pure mean-curvature flow
    void *out;
    int64_t ldu, ldf, ldo;
    int32_t h, w;
    float c_keep, c_f, c_h;
    // stacks (n images of h x w, image i at offset i * img_stride elements in u, f and out):
    // blockIdx.y is the image; lambda comes from device memory and c_h = step * lambda / 12
    int64_t img_stride;
    const float *lam;
    float step;
};

// Two adjacent elements of row `row` (already clamped or validated) starting at column x.
template <typename S, int BND, bool VEC>
__device__ __forceinline__ float2 load_pair(const S *__restrict__ row, int x, int w, bool row_ok) {
    if (BND == BND_ZERO && !row_ok) return make_float2(0.0f, 0.0f);
    if (VEC && x + 1 < w) return Store<S>::load2(row + x);
    float a, b;
    if (BND == BND_ZERO) {
        a = (x < w) ? Store<S>::load(row + x) : 0.0f;
        b = (x + 1 < w) ? Store<S>::load(row + x + 1) : 0.0f;
    } else {
        a = Store<S>::load(row + min(x, w - 1));
        b = Store<S>::load(row + min(x + 1, w - 1));
    }
    return make_float2(a, b);
}

template <typename S, int BND>
__device__ __forceinline__ float load_one(const S *__restrict__ row, int x, int w, bool row_ok) {
    if (BND == BND_ZERO) return (row_ok && x >= 0 && x < w) ? Store<S>::load(row + x) : 0.0f;
    return Store<S>::load(row + min(max(x, 0), w - 1));
}

// Row index of strip row y under the boundary rule (REPLICATE: clamped; ZERO: clamped for a
// valid address, with *ok = false marking a row of zeros).
template <int BND>
__device__ __forceinline__ int row_index(int y, int h, bool *ok) {
    *ok = (BND == BND_REPLICATE) | ((y >= 0) & (y < h));
    return min(max(y, 0), h - 1);
}

template <typename S, int BND, int MODE, bool VEC, bool STACK = false>
__global__ void __launch_bounds__(kStreamWarps * 32, 3)
    stream_kernel(const StreamParams p) {
    constexpr int R = kStreamRY;
    const int lane = threadIdx.x & 31;
    const int warp = threadIdx.x >> 5;
    const int w = p.w, h = p.h;
    float c_h = p.c_h;
    int64_t img_off = 0;
    if (STACK) {
        img_off = (int64_t)blockIdx.y * p.img_stride;
        c_h = p.step * __ldg(p.lam + blockIdx.y) / 12.0f;  // as the host computes it
    }
    // 1-D grid: block b covers row strip b / nbx and column block b % nbx (512 columns).
    const int nbx = (w + kStreamWarps * 64 - 1) / (kStreamWarps * 64);
    const int by = (int)(blockIdx.x / nbx), bx = (int)(blockIdx.x - (unsigned)by * nbx);
    const int x = ((bx * kStreamWarps + warp) * 32 + lane) * 2;
    if ((x & ~63) >= w) return;  // whole warp right of the image (warp-uniform)
    const int y0 = by * R;
    const S *__restrict__ u = static_cast<const S *>(p.u) + img_off;
    const S *__restrict__ f = p.f ? static_cast<const S *>(p.f) + img_off : nullptr;
    S *__restrict__ out = static_cast<S *>(p.out) + img_off;

    // ---- issue every load of the strip first: R + 2 rows of pairs, the two outer columns
    // (lanes 0 and 31 only) and the R rows of f
    float2 v[R + 2];
    float el[R + 2], er[R + 2];
#pragma unroll
    for (int k = 0; k < R + 2; ++k) {
        bool ok;
        const int y = row_index<BND>(y0 - 1 + k, h, &ok);
        const S *row = u + (int64_t)y * p.ldu;
        v[k] = load_pair<S, BND, VEC>(row, x, w, ok);
        el[k] = (lane == 0) ? load_one<S, BND>(row, x - 1, w, ok) : 0.0f;
        er[k] = (lane == 31) ? load_one<S, BND>(row, x + 2, w, ok) : 0.0f;
    }
    float2 g[R];
#pragma unroll
    for (int k = 0; k < R; ++k) {
        g[k] = make_float2(0.0f, 0.0f);
        if (MODE == MODE_FLOW && f != nullptr && y0 + k < h)
            g[k] = load_pair<S, BND_ZERO, VEC>(f + (int64_t)(y0 + k) * p.ldf, x, w, true);
    }

    // ---- neighbours across lanes, then the strip's R rows
    float lf[R + 2], rt[R + 2];
#pragma unroll
    for (int k = 0; k < R + 2; ++k) {
        lf[k] = __shfl_up_sync(0xffffffffu, v[k].y, 1);
        rt[k] = __shfl_down_sync(0xffffffffu, v[k].x, 1);
        if (lane == 0) lf[k] = el[k];
        if (lane == 31) rt[k] = er[k];
    }
    const float2 ch = make_float2(c_h, c_h), ck = make_float2(p.c_keep, p.c_keep);
    const float2 cf = make_float2(p.c_f, p.c_f);
#pragma unroll
    for (int k = 0; k < R; ++k) {
        const int y = y0 + k;
        // row r columns x-1 .. x+2 are (lf, v.x, v.y, rt); scalar arithmetic, since pairs of
        // adjacent columns would need register shuffling for packed operands
        const float h0 = half_laplace12(lf[k], v[k].x, v[k].y, lf[k + 1], v[k + 1].x,
                                        v[k + 1].y, lf[k + 2], v[k + 2].x, v[k + 2].y);
        const float h1 = half_laplace12(v[k].x, v[k].y, rt[k], v[k + 1].x, v[k + 1].y,
                                        rt[k + 1], v[k + 2].x, v[k + 2].y, rt[k + 2]);
        float2 o2;
        if (MODE == MODE_EVAL) {
            o2 = make_float2(ch.x * h0, ch.x * h1);
        } else {
            o2.x = fmaf(ch.x, h0, fmaf(ck.x, v[k + 1].x, cf.x * g[k].x));
            o2.y = fmaf(ch.x, h1, fmaf(ck.x, v[k + 1].y, cf.x * g[k].y));
        }
        if (y < h) {
            S *o = out + (int64_t)y * p.ldo;
            if (VEC && x + 1 < w) {
                Store<S>::store2(o + x, o2.x, o2.y);
            } else {
                if (x < w) Store<S>::store(o + x, o2.x);
                if (x + 1 < w) Store<S>::store(o + x + 1, o2.y);
            }
        }
    }
}

template <typename S, int BND, int MODE>
cudaError_t launch_stream_t(const StreamParams &p, bool vec, cudaStream_t st) {
    const int64_t nbx = (p.w + kStreamWarps * 64 - 1) / (kStreamWarps * 64);
    const int64_t nby = (p.h + kStreamRY - 1) / kStreamRY;
    if (nbx * nby > 0x7fffffffLL) return cudaErrorInvalidConfiguration;
    dim3 grid((unsigned)(nbx * nby));
    if (vec)
        stream_kernel<S, BND, MODE, true><<<grid, kStreamWarps * 32, 0, st>>>(p);
    else
        stream_kernel<S, BND, MODE, false><<<grid, kStreamWarps * 32, 0, st>>>(p);
    return cudaGetLastError();
}

template <typename S>
cudaError_t launch_stream_dtype(int mode, int bnd, const StreamParams &p, bool vec,
                                cudaStream_t st) {
    if (bnd == BND_ZERO) {
        return mode == MODE_EVAL ? launch_stream_t<S, BND_ZERO, MODE_EVAL>(p, vec, st)
                                 : launch_stream_t<S, BND_ZERO, MODE_FLOW>(p, vec, st);
    }
    return mode == MODE_EVAL ? launch_stream_t<S, BND_REPLICATE, MODE_EVAL>(p, vec, st)
                             : launch_stream_t<S, BND_REPLICATE, MODE_FLOW>(p, vec, st);
}

}  // namespace wmc
