// wmc_reduce.cu -- FP64 energies of one image:
//   E_wmc  = sum_p |H^w(U)(p)|          (the WMC regulariser of Eq. wmcr, q = 1)
//   E_data = 1/2 sum_p (U - f)^2        (the L2 data term of Eq. 1, A = I)
//   SSE    = sum_p (U - clean)^2        (for PSNR against a known clean image)
//
// The image is streamed like the single-pass kernels (a warp owns 64 columns, lanes hold column
// pairs, neighbours by warp shuffle, each thread a strip of kStreamRY rows with every load issued
// up front).  Each thread sums its 16 cells in FP32; everything after that is FP64: a fixed
// shuffle tree inside the CTA, one partial per CTA, and the last CTA to finish (ticket counter)
// adds the partials in CTA order.  The assignment and the order never change, so the result is
// bitwise reproducible.
#include "wmc_device.cuh"
#include "wmc_internal.h"
#include "wmc_stream.cuh"

namespace wmc {

int64_t energy_blocks(int32_t h, int32_t w) {
    const int64_t nbx = (w + kStreamWarps * 64 - 1) / (kStreamWarps * 64);
    const int64_t nby = (h + kStreamRY - 1) / kStreamRY;
    return nbx * nby;
}

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

template <typename S, int BND, bool VEC>
__global__ void __launch_bounds__(kStreamWarps * 32)
    energy_kernel(const S *__restrict__ u, const S *__restrict__ f, const S *__restrict__ clean,
                  int h, int w, int64_t ld, double *__restrict__ out,
                  double *__restrict__ partials, unsigned int *__restrict__ ticket) {
    constexpr int R = kStreamRY;
    const int lane = threadIdx.x & 31;
    const int warp = threadIdx.x >> 5;
    const int nbx = (w + kStreamWarps * 64 - 1) / (kStreamWarps * 64);
    const int by = (int)(blockIdx.x / nbx), bx = (int)(blockIdx.x - (unsigned)by * nbx);
    const int x = ((bx * kStreamWarps + warp) * 32 + lane) * 2;
    const int y0 = by * R;
    float s0 = 0.0f, s1 = 0.0f, s2 = 0.0f;
    if ((x & ~63) < w) {  // warp-uniform
        float2 v[R + 2];
        float el[R + 2], er[R + 2];
#pragma unroll
        for (int k = 0; k < R + 2; ++k) {
            bool ok;
            const int y = row_index<BND>(y0 - 1 + k, h, &ok);
            const S *row = u + (int64_t)y * ld;
            v[k] = load_pair<S, BND, VEC>(row, x, w, ok);
            el[k] = (lane == 0) ? load_one<S, BND>(row, x - 1, w, ok) : 0.0f;
            er[k] = (lane == 31) ? load_one<S, BND>(row, x + 2, w, ok) : 0.0f;
        }
        float2 fv[R], cv[R];
#pragma unroll
        for (int k = 0; k < R; ++k) {
            const int y = min(y0 + k, h - 1);
            fv[k] = f ? load_pair<S, BND_ZERO, VEC>(f + (int64_t)y * ld, x, w, true) : make_float2(0.f, 0.f);
            cv[k] = clean ? load_pair<S, BND_ZERO, VEC>(clean + (int64_t)y * ld, x, w, true)
                          : make_float2(0.f, 0.f);
        }
#pragma unroll
        for (int k = 0; k < R; ++k) {
            float lf = __shfl_up_sync(0xffffffffu, v[k].y, 1);
            float rt = __shfl_down_sync(0xffffffffu, v[k].x, 1);
            float lf1 = __shfl_up_sync(0xffffffffu, v[k + 1].y, 1);
            float rt1 = __shfl_down_sync(0xffffffffu, v[k + 1].x, 1);
            float lf2 = __shfl_up_sync(0xffffffffu, v[k + 2].y, 1);
            float rt2 = __shfl_down_sync(0xffffffffu, v[k + 2].x, 1);
            if (lane == 0) { lf = el[k]; lf1 = el[k + 1]; lf2 = el[k + 2]; }
            if (lane == 31) { rt = er[k]; rt1 = er[k + 1]; rt2 = er[k + 2]; }
            const int y = y0 + k;
            if (y >= h) continue;
            const float h0 = half_laplace12(lf, v[k].x, v[k].y, lf1, v[k + 1].x, v[k + 1].y, lf2,
                                            v[k + 2].x, v[k + 2].y);
            const float h1 = half_laplace12(v[k].x, v[k].y, rt, v[k + 1].x, v[k + 1].y, rt1,
                                            v[k + 2].x, v[k + 2].y, rt2);
            const bool in0 = x < w, in1 = x + 1 < w;
            if (in0) s0 += fabsf(h0) * (1.0f / 12.0f);
            if (in1) s0 += fabsf(h1) * (1.0f / 12.0f);
            if (f) {
                const float d0 = v[k + 1].x - fv[k].x, d1 = v[k + 1].y - fv[k].y;
                if (in0) s1 = fmaf(d0, d0, s1);
                if (in1) s1 = fmaf(d1, d1, s1);
            }
            if (clean) {
                const float d0 = v[k + 1].x - cv[k].x, d1 = v[k + 1].y - cv[k].y;
                if (in0) s2 = fmaf(d0, d0, s2);
                if (in1) s2 = fmaf(d1, d1, s2);
            }
        }
    }
    double acc[3] = {(double)s0, 0.5 * (double)s1, (double)s2};
    __shared__ double red[3][kStreamWarps];
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        const double t = warp_sum(acc[k]);
        if (lane == 0) red[k][warp] = t;
    }
    __syncthreads();
    __shared__ bool is_last;
    if (threadIdx.x < 3) {
        double t = 0.0;
        for (int i = 0; i < kStreamWarps; ++i) t += red[threadIdx.x][i];
        partials[(int64_t)blockIdx.x * 3 + threadIdx.x] = t;
    }
    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0) is_last = (atomicAdd(ticket, 1u) == gridDim.x - 1);
    __syncthreads();
    if (!is_last) return;
    // Last CTA: thread i sums partials i, i + 256, ... in order, then a fixed shuffle tree and
    // the 8 warp results in order -- the same order on every run.
    __threadfence();
    double a[3] = {0.0, 0.0, 0.0};
    for (unsigned b = threadIdx.x; b < gridDim.x; b += blockDim.x)
#pragma unroll
        for (int k = 0; k < 3; ++k) a[k] += __ldcg(partials + (int64_t)b * 3 + k);
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        const double t = warp_sum(a[k]);
        if (lane == 0) red[k][warp] = t;
    }
    __syncthreads();
    if (threadIdx.x < 3) {
        double t = 0.0;
        for (int i = 0; i < kStreamWarps; ++i) t += red[threadIdx.x][i];
        out[threadIdx.x] = t;
    }
}

template <typename S>
static cudaError_t launch_energy_t(const void *u, const void *f, const void *clean, int32_t h,
                                   int32_t w, int64_t ld, int bnd, double *out, void *ws,
                                   cudaStream_t st) {
    const int64_t nb = energy_blocks(h, w);
    if (nb > 0x7fffffffLL) return cudaErrorInvalidConfiguration;
    unsigned int *ticket = static_cast<unsigned int *>(ws);
    double *partials = reinterpret_cast<double *>(static_cast<char *>(ws) + 256);
    cudaError_t e = cudaMemsetAsync(ticket, 0, sizeof(unsigned int), st);
    if (e != cudaSuccess) return e;
    // 2-element loads when every row start of u, f and clean is aligned to two elements
    auto al = [&](const void *q) {
        return q == nullptr || ((uintptr_t)q % (2 * sizeof(S)) == 0 && ld % 2 == 0);
    };
    const bool vec = al(u) && al(f) && al(clean);
    const S *U = static_cast<const S *>(u), *F = static_cast<const S *>(f),
            *C = static_cast<const S *>(clean);
    const unsigned g = (unsigned)nb, b = kStreamWarps * 32;
    if (bnd == BND_ZERO) {
        if (vec) energy_kernel<S, BND_ZERO, true><<<g, b, 0, st>>>(U, F, C, h, w, ld, out, partials, ticket);
        else energy_kernel<S, BND_ZERO, false><<<g, b, 0, st>>>(U, F, C, h, w, ld, out, partials, ticket);
    } else {
        if (vec) energy_kernel<S, BND_REPLICATE, true><<<g, b, 0, st>>>(U, F, C, h, w, ld, out, partials, ticket);
        else energy_kernel<S, BND_REPLICATE, false><<<g, b, 0, st>>>(U, F, C, h, w, ld, out, partials, ticket);
    }
    return cudaGetLastError();
}

cudaError_t launch_energy(int dtype, const void *u, const void *f, const void *clean, int32_t h,
                          int32_t w, int64_t ld, int bnd, double *out, void *ws,
                          cudaStream_t st) {
    switch (dtype) {
        case 0: return launch_energy_t<float>(u, f, clean, h, w, ld, bnd, out, ws, st);
        case 1: return launch_energy_t<__nv_bfloat16>(u, f, clean, h, w, ld, bnd, out, ws, st);
        case 2: return launch_energy_t<__half>(u, f, clean, h, w, ld, bnd, out, ws, st);
        default: return cudaErrorInvalidValue;
    }
}

}  // namespace wmc
