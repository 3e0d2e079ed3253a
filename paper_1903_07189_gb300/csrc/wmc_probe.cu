// wmc_probe.cu -- a measurement utility, not part of the method: the FP32 FMA pipe's rate on this
// GPU, the denominator of the compute roofline of the temporally blocked flow kernel (which is
// bound by FP32 issue, not by memory).
//
// Every thread runs 8 independent chains of packed FP32x2 fused multiply-adds (16 lanes of work
// per iteration), enough independent work per warp to keep the pipe busy; the chains never
// converge to a constant, and one sum per thread is written so that nothing is removed.  An FMA
// counts as one lane-operation, as in the roofline of the stencil.
#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/wmc.h"

namespace {

constexpr int kProbeThreads = 256;

__global__ void __launch_bounds__(kProbeThreads) fma_probe_kernel(float *out, int32_t iters, float a, float b) {
    float2 x[8];
#pragma unroll
    for (int k = 0; k < 8; ++k) x[k] = make_float2(threadIdx.x * 1e-3f + k, blockIdx.x * 1e-3f - k);
    const float2 m = make_float2(a, a), c = make_float2(b, b);
    for (int32_t i = 0; i < iters; ++i) {
#pragma unroll
        for (int k = 0; k < 8; ++k) x[k] = __ffma2_rn(x[k], m, c);
    }
    float s = 0.0f;
#pragma unroll
    for (int k = 0; k < 8; ++k) s += x[k].x + x[k].y;
    out[blockIdx.x * kProbeThreads + threadIdx.x] = s;
}

}  // namespace

extern "C" {

int32_t wmc_probe_fma_threads(void) { return kProbeThreads; }

wmc_status_t wmc_probe_fma(float *out, int32_t blocks, int32_t iters, wmc_stream_t stream) {
    if (!out || blocks < 1 || blocks > (1 << 20) || iters < 1) return WMC_ERR_INVALID_ARG;
    // a = 1 - 2^-12, b = 2^-13: each chain contracts towards b / (1 - a) = 0.5 and stays finite
    fma_probe_kernel<<<(unsigned)blocks, kProbeThreads, 0, (cudaStream_t)stream>>>(out, iters, 1.0f - 0x1p-12f,
                                                                                   0x1p-13f);
    return cudaGetLastError() == cudaSuccess ? WMC_OK : WMC_ERR_CUDA;
}

}  // extern "C"
