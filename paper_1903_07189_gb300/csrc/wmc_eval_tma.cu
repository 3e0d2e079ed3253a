// wmc_eval_tma.cu -- one H^w evaluation pass (Eq. act) over an FP32 image whose rows start on
// 16-byte boundaries, fed by TMA.
//
// The streaming evaluation kernel issues every load of its strip before computing, so the bytes
// a thread has in flight bound it.  Here a persistent CTA (2 per SM) walks boxes of 128 x 64
// output cells through a three-stage pipeline of 136 x 66 window buffers in shared memory: while
// it computes one box, the TMA copies of its next two boxes are in flight, and no register holds
// those bytes.  Each buffer has a "full" mbarrier (the copy's bytes) and an "empty" one (one
// arrival per warp once its lanes have read the box): every warp waits for its data itself and
// releases the buffer when done, and thread 0 refills a buffer once all warps have released it,
// so the warps do not wait for each other between boxes (only border boxes under REPLICATE,
// whose ring refresh rewrites the window, take one CTA barrier).  The window geometry, the ring
// refresh, the bounded mbarrier waits and the lane layout (columns j and j + 32 of one thread
// paired in packed FP32x2 arithmetic) are those of the temporally blocked flow kernel, so every
// value equals the streaming kernel's bit for bit.
//
// Box b covers image columns x0 = 128 (b mod nbx) .. x0 + 127 and rows y0 = 64 (b div nbx) ..
// y0 + 63; its window starts at (X0, Y0) = (x0 - 4, y0 - 1): x0 - 4 keeps the TMA x coordinate on
// a 16-byte boundary, and output cell (y, x) is window cell (y - Y0, x - X0).
#include <type_traits>

#include "wmc_window.cuh"

namespace wmc {

// Set (bit 0) when a bounded wait of the evaluation kernel gave up; wmc_eval_status reads and
// clears it.
__device__ unsigned int g_eval_status;

struct EvalTmaParams {
    float *out;
    int64_t ldo;
    int32_t h, w;
    int32_t nbx, nboxes;
    float scale;
};

constexpr int kEvalBoxW = 128, kEvalBoxH = 64;
constexpr int kEvalStages = 3;
constexpr int kEvalWarps = kTileThreadsV2 / 32;
// buffer stride in floats, rounded so that every buffer starts on the 128-byte boundary a TMA
// destination needs
constexpr int kEvalBuf = (Geom<float>::LH * Geom<float>::P + 31) / 32 * 32;
static_assert((kEvalBuf * 4) % 128 == 0, "TMA destinations must be 128-byte aligned");
constexpr int kEvalX = 4;  // window column of output column x0 (and window row 1 of row y0)

template <int BND>
__global__ void __launch_bounds__(kTileThreadsV2, 2)
    eval_tma_kernel(const __grid_constant__ CUtensorMap tmap, const EvalTmaParams p) {
    using G = Geom<float>;
    constexpr int P = G::P, LW = G::LW, LH = G::LH, BUF = kEvalBuf, NS = kEvalStages;
    extern __shared__ unsigned char smem_raw[];
    __shared__ __align__(8) uint64_t full[NS], empty[NS];
    __shared__ int abort_flag;
    float *buf0 = reinterpret_cast<float *>(smem_raw + ((128u - (smem_u32(smem_raw) & 127u)) & 127u));
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int j = kEvalX + 64 * (warp & 1) + lane;  // window column of the thread's first cell
    const int ib = 1 + kRY * (warp >> 1);           // window row of its first row
    const int h = p.h, w = p.w;
    const int stride = gridDim.x;
    auto box_xy = [&](int b, int &X0, int &Y0) {
        const int by = b / p.nbx, bx = b - by * p.nbx;
        X0 = bx * kEvalBoxW - kEvalX;
        Y0 = by * kEvalBoxH - 1;
    };
    auto issue = [&](int b, int k) {  // thread 0: box b into buffer k
        int X0, Y0;
        box_xy(b, X0, Y0);
        fence_proxy_async_smem();
        mbar_expect_tx(smem_u32(&full[k]), (uint32_t)(LW * LH * 4));
        tma_load_2d(smem_u32(buf0 + k * BUF), &tmap, X0, Y0, smem_u32(&full[k]));
    };
    // thread 0's copies in flight: bit k of `pending` is set while stage k's copy has not been
    // waited for by it, bit k of `pparity` holds that copy's phase parity (a stage has at most
    // one copy in flight: it is refilled only after its previous copy was waited for)
    unsigned pending = 0, pparity = 0;
    if (tid == 0) {
        abort_flag = 0;
        for (int k = 0; k < NS; ++k) {
            mbar_init(smem_u32(&full[k]), 1);
            mbar_init(smem_u32(&empty[k]), kEvalWarps);
        }
        for (int k = 0; k < NS; ++k)
            if ((int)blockIdx.x + k * stride < p.nboxes) {
                issue(blockIdx.x + k * stride, k);
                pending |= 1u << k;  // use k of stage k: phase parity 0
            }
    }
    __syncthreads();  // the barriers are initialised before anyone waits on them
    const float2 sc = make_float2(p.scale, p.scale);
    int n = 0;
    // box coordinates stepped along with b (no division per box)
    int cbx = (int)blockIdx.x % p.nbx, cby = (int)blockIdx.x / p.nbx;
    const int sdx = stride % p.nbx, sdy = stride / p.nbx;
    for (int b = blockIdx.x; b < p.nboxes; b += stride, ++n) {
        const int k = n % NS;
        const uint32_t phase = (uint32_t)(n / NS) & 1u;
        float *buf = buf0 + k * BUF;
        // every thread waits for the copy itself (its completion makes the data visible)
        bool ok = !*static_cast<volatile int *>(&abort_flag) &&
                  mbar_wait_bounded(smem_u32(&full[k]), phase, kWaitLimitNs);
        if (tid == 0 && ok) pending &= ~(1u << k);
        if (!ok) *static_cast<volatile int *>(&abort_flag) = 1;
        const int X0 = cbx * kEvalBoxW - kEvalX, Y0 = cby * kEvalBoxH - 1;
        cbx += sdx;
        cby += sdy;
        if (cbx >= p.nbx) {
            cbx -= p.nbx;
            ++cby;
        }
        const bool border = (X0 < 0) | (Y0 < 0) | (X0 + LW > w) | (Y0 + LH > h);
        if (BND == BND_REPLICATE && border) {  // the same decision in every thread of the CTA
            const bool bad = __syncthreads_or(!ok);
            if (!bad) refresh_ring<float>(buf, X0, Y0, h, w, tid);
            __syncthreads();
            ok = !bad;
        }
        if (ok) {
            // the thread's 8 rows x 2 columns, packed FP32x2, stored where they lie in the image
            const int gx = X0 + j;
            const bool c0 = gx < w, c1 = gx + 32 < w;  // gx >= 0 always (X0 + 4 >= 0)
            const float *rp = buf + (ib - 1) * P + j;
            Row3 r0 = load_row3(rp), r1 = load_row3(rp + P);
            float *q = p.out + (int64_t)(Y0 + ib) * p.ldo + gx;
            const int64_t ldo = p.ldo;
            // a box wholly inside the image (the same for the whole CTA) stores without masks
            const bool full = (X0 + kEvalX + kEvalBoxW <= w) & (Y0 + 1 + kEvalBoxH <= h);
            auto rows = [&](auto masked) {
#pragma unroll
                for (int r = 0; r < kRY; ++r, q += ldo) {
                    const Row3 r2 = load_row3(rp + (r + 2) * P);
                    const float2 hw = half_laplace12_x2(r0.w, r0.c, r0.e, r1.w, r1.c, r1.e, r2.w, r2.c, r2.e);
                    const float2 o = __fmul2_rn(sc, hw);
                    if constexpr (decltype(masked)::value) {
                        const bool rin = Y0 + ib + r < h;
                        if (rin & c0) q[0] = o.x;
                        if (rin & c1) q[32] = o.y;
                    } else {
                        q[0] = o.x;
                        q[32] = o.y;
                    }
                    r0 = r1;
                    r1 = r2;
                }
            };
            if (full)
                rows(std::integral_constant<bool, false>{});
            else
                rows(std::integral_constant<bool, true>{});
        }
        // release the buffer: one arrival per warp, after all its lanes have read the box
        __syncwarp();
        if (lane == 0) mbar_arrive(smem_u32(&empty[k]));
        // thread 0 refills it with its box after next once every warp has released it
        if (tid == 0 && b + NS * stride < p.nboxes) {
            if (!*static_cast<volatile int *>(&abort_flag) &&
                mbar_wait_bounded(smem_u32(&empty[k]), phase, kWaitLimitNs)) {
                issue(b + NS * stride, k);
                pending |= 1u << k;
                pparity = (pparity & ~(1u << k)) | ((((uint32_t)(n / NS) + 1u) & 1u) << k);  // use n + NS
            } else {
                *static_cast<volatile int *>(&abort_flag) = 1;
            }
        }
    }
    if (tid == 0) {
        if (*static_cast<volatile int *>(&abort_flag)) atomicOr(&g_eval_status, 1u);
        // copies still in flight (after a timeout) land before the CTA's shared memory goes away
        for (int k = 0; k < NS; ++k)
            if (pending & (1u << k)) mbar_wait_bounded(smem_u32(&full[k]), (pparity >> k) & 1u, kWaitLimitNs);
    }
}

cudaError_t launch_eval_tma(const CUtensorMap *map, float *out, int64_t ldo, int32_t h, int32_t w,
                            int bnd, float scale, cudaStream_t st) {
    EvalTmaParams p;
    p.out = out;
    p.ldo = ldo;
    p.h = h;
    p.w = w;
    p.scale = scale;
    const int64_t nbx = (w + kEvalBoxW - 1) / kEvalBoxW, nby = (h + kEvalBoxH - 1) / kEvalBoxH;
    if (nbx * nby > 0x7fffffffLL) return cudaErrorInvalidConfiguration;
    p.nbx = (int32_t)nbx;
    p.nboxes = (int32_t)(nbx * nby);
    if (p.nboxes == 0) return cudaSuccess;
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    static std::atomic<int> sms[64];
    static std::atomic<uint64_t> attr_set{0};
    int nsm = sms[dev & 63].load(std::memory_order_relaxed);
    if (nsm == 0) {
        e = cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
        if (e != cudaSuccess) return e;
        sms[dev & 63].store(nsm, std::memory_order_relaxed);
    }
    const int smem = kEvalStages * kEvalBuf * 4 + 128;
    const uint64_t bit = 1ull << (dev & 63);
    if (!(attr_set.load(std::memory_order_acquire) & bit)) {
        e = cudaFuncSetAttribute(eval_tma_kernel<BND_ZERO>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
        if (e == cudaSuccess)
            e = cudaFuncSetAttribute(eval_tma_kernel<BND_REPLICATE>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     smem);
        if (e != cudaSuccess) return e;
        attr_set.fetch_or(bit, std::memory_order_release);
    }
    const int64_t grid64 = p.nboxes < 2 * nsm ? p.nboxes : 2 * nsm;
    const unsigned grid = (unsigned)grid64;
    if (bnd == BND_ZERO)
        eval_tma_kernel<BND_ZERO><<<grid, kTileThreadsV2, smem, st>>>(*map, p);
    else
        eval_tma_kernel<BND_REPLICATE><<<grid, kTileThreadsV2, smem, st>>>(*map, p);
    return cudaGetLastError();
}

cudaError_t eval_tma_status(unsigned int *word, cudaStream_t st) {
    cudaError_t e = cudaMemcpyFromSymbolAsync(word, g_eval_status, sizeof(unsigned int), 0,
                                              cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return e;
    const unsigned int zero = 0;
    e = cudaMemcpyToSymbolAsync(g_eval_status, &zero, sizeof zero, 0, cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    return e;
}

cudaError_t eval_status_word(unsigned int **word) {
    return cudaGetSymbolAddress(reinterpret_cast<void **>(word), g_eval_status);
}

}  // namespace wmc
