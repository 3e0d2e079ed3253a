// wmc_l1.cu -- one step of the L1-fidelity primal-dual iteration of Sec. V-C (A = I):
//   r = U^t - f + d^t,   d^{t+1} = clip(r, -alpha, alpha),
//   U^{t+1} = U^t + step * (lambda * H^w(U^t) - (2 d^{t+1} - d^t) / alpha).
// The step reads U^t (3x3 neighbourhood), f and d^t, and writes U^{t+1} and d^{t+1}: 20 bytes per
// pixel in FP32, so it streams like the single-pass flow kernel -- a warp owns 64 columns (lane =
// column pair, neighbours by shuffle), a thread walks a strip of kL1Rows rows with every load
// issued up front.  d is per pixel (no neighbours), so it is updated in place.  Strips of 4 rows
// with 4 CTAs per SM: 8-row strips at 3 CTAs per SM spilled 64-112 bytes (the stencil's per-row
// values shared down the strip are many registers) and ran 248 against 303 Gpix-iter/s at 4096^2.
#include "wmc_device.cuh"
#include "wmc_internal.h"
#include "wmc_stream.cuh"

namespace wmc {

constexpr int kL1Rows = 4;

template <int BND, bool VEC>
__global__ void __launch_bounds__(kStreamWarps * 32, 4)
    l1_step_kernel(const float *__restrict__ u, const float *__restrict__ f, float *__restrict__ d,
                   float *__restrict__ out, int h, int w, int64_t ld, float c_h, float c_d,
                   float alpha) {
    constexpr int R = kL1Rows;
    const int lane = threadIdx.x & 31;
    const int warp = threadIdx.x >> 5;
    const int nbx = (w + kStreamWarps * 64 - 1) / (kStreamWarps * 64);
    const int by = (int)(blockIdx.x / nbx), bx = (int)(blockIdx.x - (unsigned)by * nbx);
    const int x = ((bx * kStreamWarps + warp) * 32 + lane) * 2;
    if ((x & ~63) >= w) return;  // whole warp right of the image (warp-uniform)
    const int y0 = by * R;

    float2 v[R + 2];
    float el[R + 2], er[R + 2];
#pragma unroll
    for (int k = 0; k < R + 2; ++k) {
        bool ok;
        const int y = row_index<BND>(y0 - 1 + k, h, &ok);
        const float *row = u + (int64_t)y * ld;
        v[k] = load_pair<float, BND, VEC>(row, x, w, ok);
        el[k] = (lane == 0) ? load_one<float, BND>(row, x - 1, w, ok) : 0.0f;
        er[k] = (lane == 31) ? load_one<float, BND>(row, x + 2, w, ok) : 0.0f;
    }
    float2 fv[R], dv[R];
#pragma unroll
    for (int k = 0; k < R; ++k) {
        const bool in = y0 + k < h;
        const int64_t o = (int64_t)(in ? y0 + k : 0) * ld;
        fv[k] = load_pair<float, BND_ZERO, VEC>(f + o, x, w, in);
        dv[k] = load_pair<float, BND_ZERO, VEC>(d + o, x, w, in);
    }
    float lf[R + 2], rt[R + 2];
#pragma unroll
    for (int k = 0; k < R + 2; ++k) {
        lf[k] = __shfl_up_sync(0xffffffffu, v[k].y, 1);
        rt[k] = __shfl_down_sync(0xffffffffu, v[k].x, 1);
        if (lane == 0) lf[k] = el[k];
        if (lane == 31) rt[k] = er[k];
    }
#pragma unroll
    for (int k = 0; k < R; ++k) {
        const int y = y0 + k;
        if (y >= h) break;
        const float h0 = half_laplace12(lf[k], v[k].x, v[k].y, lf[k + 1], v[k + 1].x, v[k + 1].y,
                                        lf[k + 2], v[k + 2].x, v[k + 2].y);
        const float h1 = half_laplace12(v[k].x, v[k].y, rt[k], v[k + 1].x, v[k + 1].y, rt[k + 1],
                                        v[k + 2].x, v[k + 2].y, rt[k + 2]);
        const float u0 = v[k + 1].x, u1 = v[k + 1].y;
        const float r0 = (u0 - fv[k].x) + dv[k].x, r1 = (u1 - fv[k].y) + dv[k].y;
        const float d0 = fminf(fmaxf(r0, -alpha), alpha), d1 = fminf(fmaxf(r1, -alpha), alpha);
        const float o0 = fmaf(c_h, h0, fmaf(-c_d, fmaf(2.0f, d0, -dv[k].x), u0));
        const float o1 = fmaf(c_h, h1, fmaf(-c_d, fmaf(2.0f, d1, -dv[k].y), u1));
        const int64_t o = (int64_t)y * ld + x;
        if (VEC && x + 1 < w) {
            *reinterpret_cast<float2 *>(out + o) = make_float2(o0, o1);
            *reinterpret_cast<float2 *>(d + o) = make_float2(d0, d1);
        } else {
            if (x < w) { out[o] = o0; d[o] = d0; }
            if (x + 1 < w) { out[o + 1] = o1; d[o + 1] = d1; }
        }
    }
}

cudaError_t launch_l1_step(int bnd, const float *u, const float *f, float *d, float *out, int32_t h,
                           int32_t w, int64_t ld, float c_h, float c_d, float alpha, bool vec,
                           cudaStream_t st) {
    const int64_t nbx = (w + kStreamWarps * 64 - 1) / (kStreamWarps * 64);
    const int64_t nby = (h + kL1Rows - 1) / kL1Rows;
    if (nbx * nby > 0x7fffffffLL) return cudaErrorInvalidConfiguration;
    const unsigned g = (unsigned)(nbx * nby), b = kStreamWarps * 32;
    if (bnd == BND_ZERO) {
        if (vec) l1_step_kernel<BND_ZERO, true><<<g, b, 0, st>>>(u, f, d, out, h, w, ld, c_h, c_d, alpha);
        else l1_step_kernel<BND_ZERO, false><<<g, b, 0, st>>>(u, f, d, out, h, w, ld, c_h, c_d, alpha);
    } else {
        if (vec) l1_step_kernel<BND_REPLICATE, true><<<g, b, 0, st>>>(u, f, d, out, h, w, ld, c_h, c_d, alpha);
        else l1_step_kernel<BND_REPLICATE, false><<<g, b, 0, st>>>(u, f, d, out, h, w, ld, c_h, c_d, alpha);
    }
    return cudaGetLastError();
}

}  // namespace wmc
