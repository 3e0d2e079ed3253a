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

template <typename S, int BND, int MODE, bool VEC, bool STACK = false, int R = kStreamRY>
__global__ void __launch_bounds__(kStreamWarps * 32, R <= 8 ? 3 : 2)
    stream_kernel(const StreamParams p) {
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
        if ((MODE == MODE_FLOW || MODE == MODE_FD_FLOW) && f != nullptr && y0 + k < h)
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
        float h0, h1;
        if (MODE == MODE_FD_EVAL || MODE == MODE_FD_FLOW) {
            h0 = fd_wmc(lf[k], v[k].x, v[k].y, lf[k + 1], v[k + 1].x, v[k + 1].y, lf[k + 2],
                        v[k + 2].x, v[k + 2].y);
            h1 = fd_wmc(v[k].x, v[k].y, rt[k], v[k + 1].x, v[k + 1].y, rt[k + 1], v[k + 2].x,
                        v[k + 2].y, rt[k + 2]);
        } else {
            h0 = half_laplace12(lf[k], v[k].x, v[k].y, lf[k + 1], v[k + 1].x, v[k + 1].y,
                                lf[k + 2], v[k + 2].x, v[k + 2].y);
            h1 = half_laplace12(v[k].x, v[k].y, rt[k], v[k + 1].x, v[k + 1].y, rt[k + 1],
                                v[k + 2].x, v[k + 2].y, rt[k + 2]);
        }
        float2 o2;
        if (MODE == MODE_EVAL || MODE == MODE_FD_EVAL) {
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

// ---------------------------------------------------------------------------------------------
// FP32 images whose rows start on 16-byte boundaries: a lane holds 4 adjacent cells (one 16-byte
// access per row), a warp 128 columns, a CTA of kStream4Warps warps 512 columns, a thread a strip of
// stream4_rows<MODE, STACK>() rows.  Four cells per lane halve the shuffles and the load/store instructions per cell
// of the pair layout above; this is the form the FP32 single-pass operations take whenever the
// alignment allows it.  Every load of a strip is issued before its arithmetic, so the strip
// height sets the bytes a thread has in flight: these kernels are bound by that (evaluation moves
// 4.9 TB/s, the one-step flow, with its f rows in flight too, 7.0 TB/s at 16384^2), and 8-row
// strips (4 CTAs of 128 threads per SM, 128 registers) beat 4-row strips (6 CTAs per SM) by 3 %
// (evaluation) and 5 % (one step) at that size.  The finite-difference modes keep 4-row strips
// (their division per cell makes the 8-row form over twice as slow), and so do stacks of small
// images (32 x 512^2: 22.5 instead of 20.5 us per step with 8 rows, from the longer last wave).
#ifndef WMC_STREAM4_RY
#define WMC_STREAM4_RY 8
#endif
#ifndef WMC_STREAM4_WARPS
#define WMC_STREAM4_WARPS 4
#endif
#ifndef WMC_STREAM4_MIN_BLOCKS
#define WMC_STREAM4_MIN_BLOCKS 4
#endif
constexpr int kStream4Warps = WMC_STREAM4_WARPS;
template <int MODE>
__host__ __device__ constexpr bool stream4_fd() { return MODE == MODE_FD_EVAL || MODE == MODE_FD_FLOW; }
// 4-row strips for the finite-difference modes and for stacks of images (small images: the
// shorter strips give more CTAs and a smaller last wave)
template <int MODE, bool STACK>
__host__ __device__ constexpr bool stream4_short() { return stream4_fd<MODE>() || STACK; }
template <int MODE, bool STACK>
__host__ __device__ constexpr int stream4_rows() { return stream4_short<MODE, STACK>() ? 4 : WMC_STREAM4_RY; }
template <int MODE, bool STACK>
__host__ __device__ constexpr int stream4_min_blocks() {
    return stream4_short<MODE, STACK>() ? 6 : WMC_STREAM4_MIN_BLOCKS;
}

__device__ __forceinline__ float4 ld4(const float *p) { return *reinterpret_cast<const float4 *>(p); }

// Four adjacent elements of row `row` from column x under the boundary rule.
template <int BND>
__device__ __forceinline__ float4 load_quad(const float *__restrict__ row, int x, int w, bool row_ok) {
    if (BND == BND_ZERO && !row_ok) return make_float4(0.f, 0.f, 0.f, 0.f);
    if (x + 3 < w) return ld4(row + x);
    float4 r;
    if (BND == BND_ZERO) {
        r.x = x < w ? row[x] : 0.f;
        r.y = x + 1 < w ? row[x + 1] : 0.f;
        r.z = x + 2 < w ? row[x + 2] : 0.f;
        r.w = 0.f;
    } else {
        r.x = row[min(x, w - 1)];
        r.y = row[min(x + 1, w - 1)];
        r.z = row[min(x + 2, w - 1)];
        r.w = row[w - 1];
    }
    return r;
}

template <int MODE>
__device__ __forceinline__ float stencil4(float nw, float n, float ne, float w, float c, float e,
                                          float sw, float s, float se) {
    if (MODE == MODE_FD_EVAL || MODE == MODE_FD_FLOW) return fd_wmc(nw, n, ne, w, c, e, sw, s, se);
    return half_laplace12(nw, n, ne, w, c, e, sw, s, se);
}

template <int BND, int MODE, bool STACK = false>
__global__ void __launch_bounds__(kStream4Warps * 32, stream4_min_blocks<MODE, STACK>())
    stream4_kernel(const StreamParams p) {
    constexpr int R = stream4_rows<MODE, STACK>();
    const int lane = threadIdx.x & 31;
    const int warp = threadIdx.x >> 5;
    const int w = p.w, h = p.h;
    float c_h = p.c_h;
    int64_t img_off = 0;
    if (STACK) {
        img_off = (int64_t)blockIdx.y * p.img_stride;
        c_h = p.step * __ldg(p.lam + blockIdx.y) / 12.0f;  // as the host computes it
    }
    const int nbx = (w + kStream4Warps * 128 - 1) / (kStream4Warps * 128);
    const int by = (int)(blockIdx.x / nbx), bx = (int)(blockIdx.x - (unsigned)by * nbx);
    const int x = ((bx * kStream4Warps + warp) * 32 + lane) * 4;
    if ((x & ~127) >= w) return;  // whole warp right of the image (warp-uniform)
    const int y0 = by * R;
    const float *__restrict__ u = static_cast<const float *>(p.u) + img_off;
    const float *__restrict__ f = p.f ? static_cast<const float *>(p.f) + img_off : nullptr;
    float *__restrict__ out = static_cast<float *>(p.out) + img_off;
    constexpr bool FLOW = MODE == MODE_FLOW || MODE == MODE_FD_FLOW;

    float4 v[R + 2];
    float el[R + 2], er[R + 2];
#pragma unroll
    for (int k = 0; k < R + 2; ++k) {
        bool ok;
        const int y = row_index<BND>(y0 - 1 + k, h, &ok);
        const float *row = u + (int64_t)y * p.ldu;
        v[k] = load_quad<BND>(row, x, w, ok);
        el[k] = (lane == 0) ? load_one<float, BND>(row, x - 1, w, ok) : 0.0f;
        er[k] = (lane == 31) ? load_one<float, BND>(row, x + 4, w, ok) : 0.0f;
    }
    float4 g[R];
#pragma unroll
    for (int k = 0; k < R; ++k) {
        g[k] = make_float4(0.f, 0.f, 0.f, 0.f);
        if (FLOW && f != nullptr && y0 + k < h) g[k] = load_quad<BND_ZERO>(f + (int64_t)(y0 + k) * p.ldf, x, w, true);
    }
    float lf[R + 2], rt[R + 2];
#pragma unroll
    for (int k = 0; k < R + 2; ++k) {
        lf[k] = __shfl_up_sync(0xffffffffu, v[k].w, 1);
        rt[k] = __shfl_down_sync(0xffffffffu, v[k].x, 1);
        if (lane == 0) lf[k] = el[k];
        if (lane == 31) rt[k] = er[k];
    }
#pragma unroll
    for (int k = 0; k < R; ++k) {
        const int y = y0 + k;
        if (y >= h) break;
        const float4 a = v[k], b = v[k + 1], c = v[k + 2];
        float4 hv;
        hv.x = stencil4<MODE>(lf[k], a.x, a.y, lf[k + 1], b.x, b.y, lf[k + 2], c.x, c.y);
        hv.y = stencil4<MODE>(a.x, a.y, a.z, b.x, b.y, b.z, c.x, c.y, c.z);
        hv.z = stencil4<MODE>(a.y, a.z, a.w, b.y, b.z, b.w, c.y, c.z, c.w);
        hv.w = stencil4<MODE>(a.z, a.w, rt[k], b.z, b.w, rt[k + 1], c.z, c.w, rt[k + 2]);
        float4 o;
        if (!FLOW) {
            o = make_float4(c_h * hv.x, c_h * hv.y, c_h * hv.z, c_h * hv.w);
        } else {
            o.x = fmaf(c_h, hv.x, fmaf(p.c_keep, b.x, p.c_f * g[k].x));
            o.y = fmaf(c_h, hv.y, fmaf(p.c_keep, b.y, p.c_f * g[k].y));
            o.z = fmaf(c_h, hv.z, fmaf(p.c_keep, b.z, p.c_f * g[k].z));
            o.w = fmaf(c_h, hv.w, fmaf(p.c_keep, b.w, p.c_f * g[k].w));
        }
        float *orow = out + (int64_t)y * p.ldo;
        if (x + 3 < w) {
            *reinterpret_cast<float4 *>(orow + x) = o;
        } else {
            if (x < w) orow[x] = o.x;
            if (x + 1 < w) orow[x + 1] = o.y;
            if (x + 2 < w) orow[x + 2] = o.z;
        }
    }
}

// The 4-cell form applies: FP32, 16-byte aligned rows for u, f (if any) and out.
template <typename S>
__host__ __forceinline__ bool quad_aligned(const StreamParams &p) {
    if (sizeof(S) != 4) return false;
    auto al = [](const void *q, int64_t ld) { return q == nullptr || ((uintptr_t)q % 16 == 0 && ld % 4 == 0); };
    return al(p.u, p.ldu) && al(p.f, p.ldf) && al(p.out, p.ldo);
}

template <int BND, int MODE, bool STACK>
cudaError_t launch_stream4(const StreamParams &p, unsigned n_images, cudaStream_t st) {
    const int64_t nbx = (p.w + kStream4Warps * 128 - 1) / (kStream4Warps * 128);
    const int64_t nby = (p.h + stream4_rows<MODE, STACK>() - 1) / stream4_rows<MODE, STACK>();
    if (nbx * nby > 0x7fffffffLL) return cudaErrorInvalidConfiguration;
    dim3 grid((unsigned)(nbx * nby), n_images);
    stream4_kernel<BND, MODE, STACK><<<grid, kStream4Warps * 32, 0, st>>>(p);
    return cudaGetLastError();
}

template <typename S, int BND, int MODE>
cudaError_t launch_stream_t(const StreamParams &p, bool vec, cudaStream_t st) {
    if constexpr (sizeof(S) == 4) {
        if (quad_aligned<S>(p)) return launch_stream4<BND, MODE, false>(p, 1u, st);
    }
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

template <typename S, int BND>
cudaError_t launch_stream_mode(int mode, const StreamParams &p, bool vec, cudaStream_t st) {
    switch (mode) {
        case MODE_EVAL: return launch_stream_t<S, BND, MODE_EVAL>(p, vec, st);
        case MODE_FLOW: return launch_stream_t<S, BND, MODE_FLOW>(p, vec, st);
        case MODE_FD_EVAL: return launch_stream_t<S, BND, MODE_FD_EVAL>(p, vec, st);
        case MODE_FD_FLOW: return launch_stream_t<S, BND, MODE_FD_FLOW>(p, vec, st);
        default: return cudaErrorInvalidValue;
    }
}

template <typename S>
cudaError_t launch_stream_dtype(int mode, int bnd, const StreamParams &p, bool vec,
                                cudaStream_t st) {
    if (bnd == BND_ZERO) return launch_stream_mode<S, BND_ZERO>(mode, p, vec, st);
    return launch_stream_mode<S, BND_REPLICATE>(mode, p, vec, st);
}

}  // namespace wmc
