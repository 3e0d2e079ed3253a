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
constexpr int kStreamRY = 16;

struct StreamParams {
    const void *u;
    const void *f;  // flow only; nullptr = pure mean-curvature flow
    void *out;
    int64_t ldu, ldf, ldo;
    int32_t h, w;
    float c_keep, c_f, c_h;
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

// Columns x-1 .. x+2 of one row: .x = x-1, .y = x, .z = x+1, .w = x+2.
template <typename S, int BND, bool VEC>
__device__ __forceinline__ float4 load_row(const S *__restrict__ base, int64_t ld, int y, int h,
                                           int x, int w, int lane) {
    bool row_ok = true;
    if (BND == BND_ZERO) {
        row_ok = (y >= 0) & (y < h);
        y = min(max(y, 0), h - 1);  // keep the address valid; values are zeroed
    } else {
        y = min(max(y, 0), h - 1);
    }
    const S *row = base + (int64_t)y * ld;
    const float2 v = load_pair<S, BND, VEC>(row, x, w, row_ok);
    float left = __shfl_up_sync(0xffffffffu, v.y, 1);
    float right = __shfl_down_sync(0xffffffffu, v.x, 1);
    if (lane == 0) left = load_one<S, BND>(row, x - 1, w, row_ok);
    if (lane == 31) right = load_one<S, BND>(row, x + 2, w, row_ok);
    return make_float4(left, v.x, v.y, right);
}

template <typename S, int BND, int MODE, bool VEC>
__global__ void __launch_bounds__(kStreamWarps * 32)
    stream_kernel(const StreamParams p) {
    const int lane = threadIdx.x & 31;
    const int warp = threadIdx.x >> 5;
    const int w = p.w, h = p.h;
    // 1-D grid: block b covers row strip b / nbx and column block b % nbx (512 columns).
    const int nbx = (w + kStreamWarps * 64 - 1) / (kStreamWarps * 64);
    const int by = (int)(blockIdx.x / nbx), bx = (int)(blockIdx.x - (unsigned)by * nbx);
    const int x = ((bx * kStreamWarps + warp) * 32 + lane) * 2;
    if ((x & ~63) >= w) return;  // whole warp right of the image (warp-uniform)
    const int y0 = by * kStreamRY;
    const S *__restrict__ u = static_cast<const S *>(p.u);
    const S *__restrict__ f = static_cast<const S *>(p.f);
    S *__restrict__ out = static_cast<S *>(p.out);

    float4 r0 = load_row<S, BND, VEC>(u, p.ldu, y0 - 1, h, x, w, lane);
    float4 r1 = load_row<S, BND, VEC>(u, p.ldu, y0, h, x, w, lane);
#pragma unroll
    for (int k = 0; k < kStreamRY; ++k) {
        const int y = y0 + k;
        const float4 r2 = load_row<S, BND, VEC>(u, p.ldu, y + 1, h, x, w, lane);
        float2 g = make_float2(0.0f, 0.0f);
        if (MODE == MODE_FLOW && f != nullptr && y < h)
            g = load_pair<S, BND_ZERO, VEC>(f + (int64_t)y * p.ldf, x, w, true);
        const float h0 = half_laplace12(r0.x, r0.y, r0.z, r1.x, r1.y, r1.z, r2.x, r2.y, r2.z);
        const float h1 = half_laplace12(r0.y, r0.z, r0.w, r1.y, r1.z, r1.w, r2.y, r2.z, r2.w);
        float v0, v1;
        if (MODE == MODE_EVAL) {
            v0 = p.c_h * h0;
            v1 = p.c_h * h1;
        } else {
            v0 = fmaf(p.c_h, h0, fmaf(p.c_keep, r1.y, p.c_f * g.x));
            v1 = fmaf(p.c_h, h1, fmaf(p.c_keep, r1.z, p.c_f * g.y));
        }
        if (y < h) {
            S *o = out + (int64_t)y * p.ldo;
            if (VEC && x + 1 < w) {
                Store<S>::store2(o + x, v0, v1);
            } else {
                if (x < w) Store<S>::store(o + x, v0);
                if (x + 1 < w) Store<S>::store(o + x + 1, v1);
            }
        }
        r0 = r1;
        r1 = r2;
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
