// wmc_reduce.cu -- FP64 energies of one image:
//   E_wmc  = sum_p |H^w(U)(p)|          (the WMC regulariser of Eq. wmcr, q = 1)
//   E_data = 1/2 sum_p (U - f)^2        (the L2 data term of Eq. 1, A = I)
//   SSE    = sum_p (U - clean)^2        (for PSNR against a known clean image)
//
// A fixed grid walks the image in 16-pixel row segments.  Each thread sums a segment in FP32
// and adds the segment total to FP64 accumulators; CTAs reduce in FP64 with warp shuffles and
// write one partial each; the last CTA to finish (ticket counter) adds the partials in CTA
// order.  The grid and the assignment of segments never change, so the result is
// bitwise reproducible.
#include "wmc_device.cuh"
#include "wmc_internal.h"

namespace wmc {

constexpr int kEnergyBlocks = 608;  // 4 x 152 SMs
constexpr int kEnergyThreads = 256;
constexpr int kSeg = 16;

int energy_grid_blocks() { return kEnergyBlocks; }

template <typename S, int BND>
__device__ __forceinline__ float at(const S *u, int64_t ld, int h, int w, int y, int x) {
    if (BND == BND_ZERO) {
        if (y < 0 || y >= h || x < 0 || x >= w) return 0.0f;
    } else {
        y = min(max(y, 0), h - 1);
        x = min(max(x, 0), w - 1);
    }
    return Store<S>::load(u + (int64_t)y * ld + x);
}

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

template <typename S, int BND>
__global__ void __launch_bounds__(kEnergyThreads)
    energy_kernel(const S *__restrict__ u, const S *__restrict__ f, const S *__restrict__ clean,
                  int h, int w, int64_t ld, double *__restrict__ out,
                  double *__restrict__ partials, unsigned int *__restrict__ ticket) {
    const int64_t segs_per_row = (w + kSeg - 1) / kSeg;
    const int64_t nseg = (int64_t)h * segs_per_row;
    double acc[3] = {0.0, 0.0, 0.0};
    for (int64_t t = blockIdx.x * (int64_t)kEnergyThreads + threadIdx.x; t < nseg;
         t += (int64_t)kEnergyBlocks * kEnergyThreads) {
        const int y = (int)(t / segs_per_row);
        const int xb = (int)(t - (int64_t)y * segs_per_row) * kSeg;
        const int xe = min(xb + kSeg, w);
        float s0 = 0.0f, s1 = 0.0f, s2 = 0.0f;
        for (int x = xb; x < xe; ++x) {
            const float c = at<S, BND>(u, ld, h, w, y, x);
            const float h12 = half_laplace12(
                at<S, BND>(u, ld, h, w, y - 1, x - 1), at<S, BND>(u, ld, h, w, y - 1, x),
                at<S, BND>(u, ld, h, w, y - 1, x + 1), at<S, BND>(u, ld, h, w, y, x - 1), c,
                at<S, BND>(u, ld, h, w, y, x + 1), at<S, BND>(u, ld, h, w, y + 1, x - 1),
                at<S, BND>(u, ld, h, w, y + 1, x), at<S, BND>(u, ld, h, w, y + 1, x + 1));
            s0 += fabsf(h12) * (1.0f / 12.0f);
            if (f) {
                const float d = c - Store<S>::load(f + (int64_t)y * ld + x);
                s1 = fmaf(d, d, s1);
            }
            if (clean) {
                const float d = c - Store<S>::load(clean + (int64_t)y * ld + x);
                s2 = fmaf(d, d, s2);
            }
        }
        acc[0] += (double)s0;
        acc[1] += 0.5 * (double)s1;
        acc[2] += (double)s2;
    }
    __shared__ double red[3][kEnergyThreads / 32];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        const double v = warp_sum(acc[k]);
        if (lane == 0) red[k][wid] = v;
    }
    __syncthreads();
    __shared__ bool is_last;
    if (threadIdx.x < 3) {
        double v = 0.0;
        for (int i = 0; i < kEnergyThreads / 32; ++i) v += red[threadIdx.x][i];
        partials[blockIdx.x * 3 + threadIdx.x] = v;
    }
    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0) is_last = (atomicAdd(ticket, 1u) == kEnergyBlocks - 1);
    __syncthreads();
    if (is_last && threadIdx.x < 3) {
        __threadfence();
        double v = 0.0;
        for (int b = 0; b < kEnergyBlocks; ++b)
            v += *((volatile double *)partials + b * 3 + threadIdx.x);
        out[threadIdx.x] = v;
    }
}

template <typename S>
static cudaError_t launch_energy_t(const void *u, const void *f, const void *clean, int32_t h,
                                   int32_t w, int64_t ld, int bnd, double *out, void *ws,
                                   cudaStream_t st) {
    double *partials = static_cast<double *>(ws);
    unsigned int *ticket = reinterpret_cast<unsigned int *>(partials + 3 * kEnergyBlocks);
    cudaError_t e = cudaMemsetAsync(ticket, 0, sizeof(unsigned int), st);
    if (e != cudaSuccess) return e;
    if (bnd == BND_ZERO)
        energy_kernel<S, BND_ZERO><<<kEnergyBlocks, kEnergyThreads, 0, st>>>(
            static_cast<const S *>(u), static_cast<const S *>(f), static_cast<const S *>(clean), h,
            w, ld, out, partials, ticket);
    else
        energy_kernel<S, BND_REPLICATE><<<kEnergyBlocks, kEnergyThreads, 0, st>>>(
            static_cast<const S *>(u), static_cast<const S *>(f), static_cast<const S *>(clean), h,
            w, ld, out, partials, ticket);
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
