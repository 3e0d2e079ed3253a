// wmc_reduce.cu -- FP64 energies of one image:
//   E_wmc  = sum_p |H^w(U)(p)|          (the WMC regulariser of Eq. wmcr, q = 1)
//   E_data = 1/2 sum_p (U - f)^2        (the L2 data term of Eq. 1, A = I)
//   SSE    = sum_p (U - clean)^2        (for PSNR against a known clean image)
//
// The image is streamed like the single-pass kernels: lanes hold 2 adjacent cells (any type) or 4
// (FP32 rows aligned to 16 bytes), neighbours come by warp shuffle, and each thread takes a strip
// of rows with every load issued up front, summing its 16 cells in FP32.  A CTA walks a fixed run
// of strips and adds each strip's sums into double-float (hi + lo) accumulators; a shuffle tree
// of double-float adds per warp, then FP64: the warps in order, one partial per CTA, and the last
// CTA to finish (ticket counter) adds the partials in CTA order.  The assignment and the order
// never change, so the result is bitwise reproducible.
#include <atomic>

#include "wmc_device.cuh"
#include "wmc_internal.h"
#include "wmc_stream.cuh"
#include <type_traits>

#include "wmc_window.cuh"

namespace wmc {

// Pair layout: a unit of work is one strip, a CTA's 512 columns times kStreamRY rows.  The grid
// is a pure function of the image size -- at most kEnergyCTAs CTAs (2 resident per SM on 152
// SMs, one wave) -- and CTA b walks the units [b*U/N, (b+1)*U/N) in order.
// Four cells per lane: a CTA owns 1024 columns and a band of rows (a multiple of 4), and its
// threads march down the band.  Either way the summation order never changes.
#ifndef WMC_ENERGY_MIN_BLOCKS
#define WMC_ENERGY_MIN_BLOCKS 2
#endif
constexpr int kEnergyCTAs = WMC_ENERGY_MIN_BLOCKS * 152;

static int64_t energy_grid(int32_t h, int32_t w) {
    const int64_t u = (int64_t)((w + kStreamWarps * 64 - 1) / (kStreamWarps * 64)) *
                      ((h + kStreamRY - 1) / kStreamRY);
    return u < kEnergyCTAs ? u : kEnergyCTAs;
}

struct MarchGeom {
    int nbx, band_rows, nbands;
};

__host__ __device__ __forceinline__ MarchGeom march_geom(int32_t h, int32_t w) {
    MarchGeom g;
    g.nbx = (int)(((int64_t)w + kStreamWarps * 128 - 1) / (kStreamWarps * 128));
    int64_t nb = kEnergyCTAs / g.nbx;
    if (nb < 1) nb = 1;
    const int64_t br = (((int64_t)h + nb - 1) / nb + 3) & ~(int64_t)3;
    g.band_rows = (int)br;
    g.nbands = (int)(((int64_t)h + br - 1) / br);
    return g;
}

// TMA-fed kernel: boxes of 128 x 64 cells, at most kEnergyTmaCTAs persistent CTAs (one per SM on
// 152 SMs); the grid is a pure function of the image size, so the summation order is too.
constexpr int kEBoxW = 128, kEBoxH = 64, kEnergyTmaCTAs = 152;

static int64_t energy_tma_grid(int32_t h, int32_t w) {
    const int64_t nb = (((int64_t)w + kEBoxW - 1) / kEBoxW) * (((int64_t)h + kEBoxH - 1) / kEBoxH);
    return nb < kEnergyTmaCTAs ? nb : kEnergyTmaCTAs;
}

int64_t energy_blocks(int32_t h, int32_t w) {
    const MarchGeom g = march_geom(h, w);
    int64_t a = energy_grid(h, w), b = (int64_t)g.nbx * g.nbands;
    if (b > a) a = b;
    b = energy_tma_grid(h, w);
    return a > b ? a : b;
}

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// Double-float accumulator: the unevaluated sum hi + lo.  Adding a float is exact in (s, e) by
// Knuth's TwoSum; the rounding errors collect in lo.  All summands here are >= 0, so no
// cancellation occurs and the accumulated value keeps about 44 bits.  GB300 issues FP64 at a
// small fraction of its FP32 rate, so only the last steps of the reduction run in FP64.
struct DF {
    float hi, lo;
};

__device__ __forceinline__ void two_sum(float a, float b, float &s, float &e) {
    s = __fadd_rn(a, b);
    const float bb = __fsub_rn(s, a);
    e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
}

__device__ __forceinline__ void df_add(DF &a, float x) {
    float s, e;
    two_sum(a.hi, x, s, e);
    a.hi = s;
    a.lo = __fadd_rn(a.lo, e);
}

__device__ __forceinline__ DF df_merge(DF a, DF b) {
    float s, e;
    two_sum(a.hi, b.hi, s, e);
    const float lo = __fadd_rn(__fadd_rn(a.lo, b.lo), e);
    const float hi = __fadd_rn(s, lo);  // renormalise (Fast2Sum: |s| >= |lo|)
    return {hi, __fsub_rn(lo, __fsub_rn(hi, s))};
}

__device__ __forceinline__ DF df_warp_sum(DF v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        DF t;
        t.hi = __shfl_xor_sync(0xffffffffu, v.hi, o);
        t.lo = __shfl_xor_sync(0xffffffffu, v.lo, o);
        // lanes l and l^o merge the same two operands in the same order
        v = ((threadIdx.x & o) == 0) ? df_merge(v, t) : df_merge(t, v);
    }
    return v;
}

// Thread sums (12 |H^w|, the squared data residual, the squared error) as double-float pairs:
// a fixed shuffle tree per warp, one FP64 value per warp (hi + lo), the 8 warps in order, one
// partial per CTA, and the last CTA to finish (ticket counter) adds the partials in CTA order.
template <int NW = kStreamWarps>  // warps per CTA
__device__ __forceinline__ void energy_reduce(const DF (&acc)[3], double *__restrict__ out,
                                              double *__restrict__ partials,
                                              unsigned int *__restrict__ ticket) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    __shared__ double red[3][NW];
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        const DF t = df_warp_sum(acc[k]);
        if (lane == 0) red[k][warp] = (double)t.hi + (double)t.lo;
    }
    __syncthreads();
    __shared__ bool is_last;
    if (threadIdx.x < 3) {
        double t = 0.0;
        for (int i = 0; i < NW; ++i) t += red[threadIdx.x][i];
        // the thread sums hold 12 |H^w| and (U - f)^2: scale once, in FP64
        partials[(int64_t)blockIdx.x * 3 + threadIdx.x] =
            threadIdx.x == 0 ? t / 12.0 : threadIdx.x == 1 ? 0.5 * t : t;
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
    __syncthreads();  // red[] is reused
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        const double t = warp_sum(a[k]);
        if (lane == 0) red[k][warp] = t;
    }
    __syncthreads();
    if (threadIdx.x < 3) {
        double t = 0.0;
        for (int i = 0; i < NW; ++i) t += red[threadIdx.x][i];
        out[threadIdx.x] = t;
    }
}

// One strip in the pair layout: a lane holds 2 adjacent cells, a warp 64 columns, the thread
// kStreamRY rows (16 cells, summed in FP32).  Loads are issued before any arithmetic.
template <typename S, int BND, bool VEC>
__device__ __forceinline__ void energy_strip_pair(const S *__restrict__ u, const S *__restrict__ f,
                                                  const S *__restrict__ clean, int h, int w,
                                                  int64_t ld, int bx, int by, float (&s)[3]) {
    constexpr int R = kStreamRY;
    const int lane = threadIdx.x & 31;
    const int warp = threadIdx.x >> 5;
    const int x = ((bx * kStreamWarps + warp) * 32 + lane) * 2;
    const int y0 = by * R;
    if ((x & ~63) >= w) return;  // warp-uniform
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
        if (y0 + k >= h) continue;
        const float h0 = half_laplace12(lf, v[k].x, v[k].y, lf1, v[k + 1].x, v[k + 1].y, lf2,
                                        v[k + 2].x, v[k + 2].y);
        const float h1 = half_laplace12(v[k].x, v[k].y, rt, v[k + 1].x, v[k + 1].y, rt1,
                                        v[k + 2].x, v[k + 2].y, rt2);
        const bool in0 = x < w, in1 = x + 1 < w;
        if (in0) s[0] += fabsf(h0);
        if (in1) s[0] += fabsf(h1);
        if (f) {
            const float d0 = v[k + 1].x - fv[k].x, d1 = v[k + 1].y - fv[k].y;
            if (in0) s[1] = fmaf(d0, d0, s[1]);
            if (in1) s[1] = fmaf(d1, d1, s[1]);
        }
        if (clean) {
            const float d0 = v[k + 1].x - cv[k].x, d1 = v[k + 1].y - cv[k].y;
            if (in0) s[2] = fmaf(d0, d0, s[2]);
            if (in1) s[2] = fmaf(d1, d1, s[2]);
        }
    }
}

// Four cells per lane (FP32, 16-byte aligned rows): a warp holds 128 columns and its threads
// march down the CTA's band with a three-row window (rows y-1, y, y+1) in registers, loading
// the next 4 rows of U (and of f, clean) before computing any of them.  Each group of 4 rows
// (16 cells) is summed in FP32 and added into the double-float accumulators.  HF, HC: f, clean
// given (the unused terms cost no registers).
template <int BND, bool HF, bool HC>
__global__ void __launch_bounds__(kStreamWarps * 32, WMC_ENERGY_MIN_BLOCKS)
    energy_march_kernel(const float *__restrict__ u, const float *__restrict__ f,
                        const float *__restrict__ clean, int h, int w, int64_t ld,
                        double *__restrict__ out, double *__restrict__ partials,
                        unsigned int *__restrict__ ticket) {
    const MarchGeom g = march_geom(h, w);
    const int band = (int)(blockIdx.x / g.nbx), bx = (int)(blockIdx.x - (unsigned)band * g.nbx);
    const int lane = threadIdx.x & 31;
    const int warp = threadIdx.x >> 5;
    const int x = ((bx * kStreamWarps + warp) * 32 + lane) * 4;
    const int yb = band * g.band_rows, ye = min(yb + g.band_rows, h);
    DF acc[3] = {{0.f, 0.f}, {0.f, 0.f}, {0.f, 0.f}};
    auto load_row = [&](int y, float4 &v, float &el, float &er) {
        bool ok;
        const int yy = row_index<BND>(y, h, &ok);
        const float *row = u + (int64_t)yy * ld;
        v = load_quad<BND>(row, x, w, ok);
        el = (lane == 0) ? load_one<float, BND>(row, x - 1, w, ok) : 0.0f;
        er = (lane == 31) ? load_one<float, BND>(row, x + 4, w, ok) : 0.0f;
    };
    // left neighbour of the lane's first cell, right neighbour of its last
    auto sides = [&](const float4 &v, float el, float er, float &l, float &r) {
        l = __shfl_up_sync(0xffffffffu, v.w, 1);
        r = __shfl_down_sync(0xffffffffu, v.x, 1);
        if (lane == 0) l = el;
        if (lane == 31) r = er;
    };
    if ((x & ~127) < w) {  // warp-uniform
        float4 top, mid;
        float tl, tr, ml, mr;
        {
            float e0, e1;
            load_row(yb - 1, top, e0, e1);
            sides(top, e0, e1, tl, tr);
            load_row(yb, mid, e0, e1);
            sides(mid, e0, e1, ml, mr);
        }
        for (int y = yb; y < ye; y += 4) {
            float4 nv[4], fv[4], cv[4];
            float nel[4], ner[4];
#pragma unroll
            for (int k = 0; k < 4; ++k) load_row(y + 1 + k, nv[k], nel[k], ner[k]);
#pragma unroll
            for (int k = 0; k < 4; ++k) {
                const int yy = min(y + k, h - 1);
                fv[k] = HF ? load_quad<BND_ZERO>(f + (int64_t)yy * ld, x, w, true) : make_float4(0.f, 0.f, 0.f, 0.f);
                cv[k] = HC ? load_quad<BND_ZERO>(clean + (int64_t)yy * ld, x, w, true) : make_float4(0.f, 0.f, 0.f, 0.f);
            }
            float s[3] = {0.f, 0.f, 0.f};
#pragma unroll
            for (int k = 0; k < 4; ++k) {
                float bl, br;
                sides(nv[k], nel[k], ner[k], bl, br);
                if (y + k < ye) {  // uniform over the CTA
                    const float4 a = top, b = mid, c = nv[k];
                    const float hs[4] = {half_laplace12(tl, a.x, a.y, ml, b.x, b.y, bl, c.x, c.y),
                                         half_laplace12(a.x, a.y, a.z, b.x, b.y, b.z, c.x, c.y, c.z),
                                         half_laplace12(a.y, a.z, a.w, b.y, b.z, b.w, c.y, c.z, c.w),
                                         half_laplace12(a.z, a.w, tr, b.z, b.w, mr, c.z, c.w, br)};
                    const float uu[4] = {b.x, b.y, b.z, b.w};
                    const float ff[4] = {fv[k].x, fv[k].y, fv[k].z, fv[k].w};
                    const float cc[4] = {cv[k].x, cv[k].y, cv[k].z, cv[k].w};
                    if (x + 3 < w) {  // every lane but those at the right edge
#pragma unroll
                        for (int q = 0; q < 4; ++q) s[0] += fabsf(hs[q]);
                        if (HF) {
#pragma unroll
                            for (int q = 0; q < 4; ++q) {
                                const float d = uu[q] - ff[q];
                                s[1] = fmaf(d, d, s[1]);
                            }
                        }
                        if (HC) {
#pragma unroll
                            for (int q = 0; q < 4; ++q) {
                                const float d = uu[q] - cc[q];
                                s[2] = fmaf(d, d, s[2]);
                            }
                        }
                    } else {
#pragma unroll
                        for (int q = 0; q < 4; ++q) {
                            if (x + q >= w) continue;
                            s[0] += fabsf(hs[q]);
                            const float d1 = uu[q] - ff[q], d2 = uu[q] - cc[q];
                            if (HF) s[1] = fmaf(d1, d1, s[1]);
                            if (HC) s[2] = fmaf(d2, d2, s[2]);
                        }
                    }
                }
                top = mid;
                tl = ml;
                tr = mr;
                mid = nv[k];
                ml = bl;
                mr = br;
            }
#pragma unroll
            for (int k = 0; k < 3; ++k) df_add(acc[k], s[k]);
        }
    }
    energy_reduce(acc, out, partials, ticket);
}

// Pair layout (any storage type): each strip's FP32 sums enter the thread's double-float
// accumulators.
template <typename S, int BND, bool VEC>
__global__ void __launch_bounds__(kStreamWarps * 32, 2)
    energy_kernel(const S *__restrict__ u, const S *__restrict__ f, const S *__restrict__ clean,
                  int h, int w, int64_t ld, double *__restrict__ out,
                  double *__restrict__ partials, unsigned int *__restrict__ ticket) {
    const int nbx = (w + kStreamWarps * 64 - 1) / (kStreamWarps * 64);
    const int64_t units = (int64_t)nbx * ((h + kStreamRY - 1) / kStreamRY);
    const int64_t u0 = units * blockIdx.x / gridDim.x, u1 = units * (blockIdx.x + 1) / gridDim.x;
    DF acc[3] = {{0.f, 0.f}, {0.f, 0.f}, {0.f, 0.f}};
    for (int64_t un = u0; un < u1; ++un) {
        const int by = (int)(un / nbx), bx = (int)(un - (int64_t)by * nbx);
        float s[3] = {0.f, 0.f, 0.f};
        energy_strip_pair<S, BND, VEC>(u, f, clean, h, w, ld, bx, by, s);
#pragma unroll
        for (int k = 0; k < 3; ++k) df_add(acc[k], s[k]);
    }
    energy_reduce(acc, out, partials, ticket);
}

// FP32 images that TMA can read: persistent CTAs (one per SM, 512 threads) walk boxes of 128 x 64
// cells.  A buffer holds U's 136 x 66 window (origin (x0 - 4, y0 - 1), the flow kernel's, ring
// refreshed for REPLICATE border boxes) and dense 128 x 64 boxes of f and clean; two buffers per
// CTA, each with a "full" mbarrier (the copies' bytes) and an "empty" one (one arrival per warp
// once it has read the box), so the next box's copies are in flight while the current box is
// summed and the warps do not wait for each other between boxes (border boxes under REPLICATE
// take one CTA barrier for the ring refresh).  A thread takes columns j and j + 32 of 8 rows
// (the packed FP32x2 stencil, the magnitude of the selection only), sums its 16 cells in FP32 per
// box and adds those sums into its double-float accumulators.  (1024 threads of 4 rows each,
// for more warps per SM, measured slower: 54.8 against 44.5 us at 4096^2.)  A window wait that runs out turns
// the CTA's partial sums into NaN (after a bounded wait for its copies in flight), so the
// energies come out NaN instead of wrong.
constexpr int kEUBuf = (Geom<float>::LH * Geom<float>::P + 31) / 32 * 32;  // U window, floats
constexpr int kEFBuf = kEBoxW * kEBoxH;                                     // f or clean box
constexpr int kEThreads = 512, kERY = 8, kEWarps = kEThreads / 32;
static_assert((kEUBuf * 4) % 128 == 0 && (kEFBuf * 4) % 128 == 0, "TMA destinations 128-byte aligned");
static_assert(kERY * (kEWarps / 2) == kEBoxH, "2 warps across, kEWarps / 2 warps down cover a box");

template <bool HF, bool HC>
__host__ __device__ constexpr int energy_tma_buf() { return kEUBuf + (HF ? kEFBuf : 0) + (HC ? kEFBuf : 0); }

template <int BND, bool HF, bool HC>
__global__ void __launch_bounds__(kEThreads, 1)
    energy_tma_kernel(const __grid_constant__ CUtensorMap umap, const __grid_constant__ CUtensorMap fmap,
                      const __grid_constant__ CUtensorMap cmap, int h, int w, double *__restrict__ out,
                      double *__restrict__ partials, unsigned int *__restrict__ ticket) {
    using G = Geom<float>;
    constexpr int P = G::P, LW = G::LW, LH = G::LH, NB = energy_tma_buf<HF, HC>();
    constexpr uint32_t BYTES = (uint32_t)(LW * LH + (HF ? kEFBuf : 0) + (HC ? kEFBuf : 0)) * 4u;
    extern __shared__ unsigned char smem_raw[];
    __shared__ __align__(8) uint64_t full[2], empty[2];
    __shared__ int abort_flag;
    float *buf0 = reinterpret_cast<float *>(smem_raw + ((128u - (smem_u32(smem_raw) & 127u)) & 127u));
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int j = 4 + 64 * (warp & 1) + lane;  // window column of the thread's first cell
    const int ib = 1 + kERY * (warp >> 1);      // window row of its first row
    const int nbx = (w + kEBoxW - 1) / kEBoxW;
    const int nboxes = nbx * ((h + kEBoxH - 1) / kEBoxH);
    const int stride = gridDim.x;
    auto issue = [&](int b, int k) {  // thread 0: the copies of box b into buffer k
        const int by = b / nbx, bx = b - by * nbx;
        float *bk = buf0 + k * NB;
        fence_proxy_async_smem();
        mbar_expect_tx(smem_u32(&full[k]), BYTES);
        tma_load_2d(smem_u32(bk), &umap, bx * kEBoxW - 4, by * kEBoxH - 1, smem_u32(&full[k]));
        if (HF) tma_load_2d(smem_u32(bk + kEUBuf), &fmap, bx * kEBoxW, by * kEBoxH, smem_u32(&full[k]));
        if (HC)
            tma_load_2d(smem_u32(bk + kEUBuf + (HF ? kEFBuf : 0)), &cmap, bx * kEBoxW, by * kEBoxH,
                        smem_u32(&full[k]));
    };
    // thread 0's copies in flight (bit k of `pending`) and their phase parities (`pparity`)
    unsigned pending = 0, pparity = 0;
    if (tid == 0) {
        abort_flag = 0;
        for (int k = 0; k < 2; ++k) {
            mbar_init(smem_u32(&full[k]), 1);
            mbar_init(smem_u32(&empty[k]), kEWarps);
        }
        for (int k = 0; k < 2; ++k)
            if ((int)blockIdx.x + k * stride < nboxes) {
                issue(blockIdx.x + k * stride, k);
                pending |= 1u << k;
            }
    }
    __syncthreads();  // the barriers are initialised before anyone waits on them
    volatile int *abort_v = &abort_flag;
    DF acc[3] = {{0.f, 0.f}, {0.f, 0.f}, {0.f, 0.f}};
    int n = 0;
    // box coordinates stepped along with b (no division per box)
    int cbx = (int)blockIdx.x % nbx, cby = (int)blockIdx.x / nbx;
    const int sdx = stride % nbx, sdy = stride / nbx;
    for (int b = blockIdx.x; b < nboxes; b += stride, ++n) {
        const int k = n & 1;
        const uint32_t phase = (uint32_t)(n >> 1) & 1u;
        const float *bu = buf0 + k * NB;
        const float *bf = bu + kEUBuf, *bc = bu + kEUBuf + (HF ? kEFBuf : 0);
        bool ok = !*abort_v && mbar_wait_bounded(smem_u32(&full[k]), phase, kWaitLimitNs);
        if (tid == 0 && ok) pending &= ~(1u << k);
        if (!ok) *abort_v = 1;
        const int bx = cbx, by = cby;
        cbx += sdx;
        cby += sdy;
        if (cbx >= nbx) {
            cbx -= nbx;
            ++cby;
        }
        const int X0 = bx * kEBoxW - 4, Y0 = by * kEBoxH - 1;
        const bool border = (X0 < 0) | (Y0 < 0) | (X0 + LW > w) | (Y0 + LH > h);
        if (BND == BND_REPLICATE && border) {  // the same decision in every thread of the CTA
            const bool bad = __syncthreads_or(!ok);
            if (!bad) refresh_ring<float, G::LH, kEThreads>(const_cast<float *>(bu), X0, Y0, h, w, tid);
            __syncthreads();
            ok = !bad;
        }
        if (ok) {
            const int gx = X0 + j;
            const bool c0 = gx < w, c1 = gx + 32 < w;
            const float *rp = bu + (ib - 1) * P + j;
            const int fo = (ib - 1) * kEBoxW + (j - 4);  // box offset of the thread's first cell
            Row3 r0 = load_row3(rp), r1 = load_row3(rp + P);
            // per-lane sums of the thread's two columns (8 cells each), as FP32x2 pairs
            float2 s2[3] = {{0.f, 0.f}, {0.f, 0.f}, {0.f, 0.f}};
            // a box wholly inside the image (the same for the whole CTA) needs no cell masks
            const bool full = (bx + 1) * kEBoxW <= w && (by + 1) * kEBoxH <= h;
            auto rows = [&](auto masked) {
#pragma unroll
                for (int r = 0; r < kERY; ++r) {
                    const Row3 r2 = load_row3(rp + (r + 2) * P);
                    float2 a12 = abs_half_laplace12_x2(r0.w, r0.c, r0.e, r1.w, r1.c, r1.e, r2.w, r2.c, r2.e);
                    float2 df = make_float2(0.f, 0.f), dc = make_float2(0.f, 0.f);
                    if (HF) df = sub2(r1.c, make_float2(bf[fo + r * kEBoxW], bf[fo + r * kEBoxW + 32]));
                    if (HC) dc = sub2(r1.c, make_float2(bc[fo + r * kEBoxW], bc[fo + r * kEBoxW + 32]));
                    if constexpr (decltype(masked)::value) {
                        const bool rin = Y0 + ib + r < h;
                        const bool in0 = rin & c0, in1 = rin & c1;
                        a12 = make_float2(in0 ? a12.x : 0.f, in1 ? a12.y : 0.f);
                        df = make_float2(in0 ? df.x : 0.f, in1 ? df.y : 0.f);
                        dc = make_float2(in0 ? dc.x : 0.f, in1 ? dc.y : 0.f);
                    }
                    s2[0] = __fadd2_rn(s2[0], a12);
                    if (HF) s2[1] = __ffma2_rn(df, df, s2[1]);
                    if (HC) s2[2] = __ffma2_rn(dc, dc, s2[2]);
                    r0 = r1;
                    r1 = r2;
                }
            };
            if (full)
                rows(std::integral_constant<bool, false>{});
            else
                rows(std::integral_constant<bool, true>{});
            const float s[3] = {s2[0].x + s2[0].y, s2[1].x + s2[1].y, s2[2].x + s2[2].y};
#pragma unroll
            for (int q = 0; q < 3; ++q) df_add(acc[q], s[q]);
        }
        // release the buffer: one arrival per warp, after all its lanes have read the box
        __syncwarp();
        if (lane == 0) mbar_arrive(smem_u32(&empty[k]));
        // thread 0 refills it with its box after next once every warp has released it
        if (tid == 0 && b + 2 * stride < nboxes) {
            if (!*abort_v && mbar_wait_bounded(smem_u32(&empty[k]), phase, kWaitLimitNs)) {
                issue(b + 2 * stride, k);
                pending |= 1u << k;
                pparity = (pparity & ~(1u << k)) | ((((uint32_t)(n >> 1) + 1u) & 1u) << k);
            } else {
                *abort_v = 1;
            }
        }
    }
    if (tid == 0)  // copies still in flight (after a timeout) land before the CTA's shared memory goes away
        for (int k = 0; k < 2; ++k)
            if (pending & (1u << k)) mbar_wait_bounded(smem_u32(&full[k]), (pparity >> k) & 1u, kWaitLimitNs);
    __syncthreads();
    if (*abort_v) {  // the energies come out NaN instead of wrong
        const float nan = __int_as_float(0x7fc00000);
        for (int q = 0; q < 3; ++q) acc[q] = {nan, 0.f};
    }
    energy_reduce<kEWarps>(acc, out, partials, ticket);
}

void energy_tma_box(int *bw, int *bh) {
    *bw = kEBoxW;
    *bh = kEBoxH;
}

cudaError_t launch_energy_tma(const CUtensorMap *maps, bool has_f, bool has_clean, int32_t h, int32_t w,
                              int bnd, double *out, void *ws, cudaStream_t st) {
    unsigned int *ticket = static_cast<unsigned int *>(ws);
    double *partials = reinterpret_cast<double *>(static_cast<char *>(ws) + 256);
    cudaError_t e = cudaMemsetAsync(ticket, 0, sizeof(unsigned int), st);
    if (e != cudaSuccess) return e;
    const unsigned g = (unsigned)energy_tma_grid(h, w), b = kEThreads;
    // one shared-memory size for every instance: two buffers of the largest kind
    const int smem = 2 * energy_tma_buf<true, true>() * 4 + 128;
    int dev = 0;
    e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    static std::atomic<uint64_t> attr_set{0};
    const uint64_t bit = 1ull << (dev & 63);
    auto go = [&](auto kern) -> cudaError_t {
        kern<<<g, b, smem, st>>>(maps[0], maps[1], maps[2], h, w, out, partials, ticket);
        return cudaGetLastError();
    };
#define WMC_ENERGY_TMA_KERNELS(B)                                                                       \
    energy_tma_kernel<B, false, false>, energy_tma_kernel<B, true, false>, energy_tma_kernel<B, false, true>, \
        energy_tma_kernel<B, true, true>
    if (!(attr_set.load(std::memory_order_acquire) & bit)) {
        void (*ks[8])(CUtensorMap, CUtensorMap, CUtensorMap, int, int, double *, double *, unsigned int *) = {
            WMC_ENERGY_TMA_KERNELS(BND_REPLICATE), WMC_ENERGY_TMA_KERNELS(BND_ZERO)};
        for (auto kf : ks) {
            e = cudaFuncSetAttribute(kf, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
            if (e != cudaSuccess) return e;
        }
        attr_set.fetch_or(bit, std::memory_order_release);
    }
#undef WMC_ENERGY_TMA_KERNELS
    const int sel = (bnd == BND_ZERO ? 4 : 0) | (has_f ? 1 : 0) | (has_clean ? 2 : 0);
    switch (sel) {
        case 0: return go(energy_tma_kernel<BND_REPLICATE, false, false>);
        case 1: return go(energy_tma_kernel<BND_REPLICATE, true, false>);
        case 2: return go(energy_tma_kernel<BND_REPLICATE, false, true>);
        case 3: return go(energy_tma_kernel<BND_REPLICATE, true, true>);
        case 4: return go(energy_tma_kernel<BND_ZERO, false, false>);
        case 5: return go(energy_tma_kernel<BND_ZERO, true, false>);
        case 6: return go(energy_tma_kernel<BND_ZERO, false, true>);
        default: return go(energy_tma_kernel<BND_ZERO, true, true>);
    }
}

template <typename S>
static cudaError_t launch_energy_t(const void *u, const void *f, const void *clean, int32_t h,
                                   int32_t w, int64_t ld, int bnd, double *out, void *ws,
                                   cudaStream_t st) {
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
    const unsigned b = kStreamWarps * 32;
    if constexpr (sizeof(S) == 4) {
        auto al16 = [&](const void *q) { return q == nullptr || ((uintptr_t)q % 16 == 0 && ld % 4 == 0); };
        if (al16(u) && al16(f) && al16(clean)) {
            const MarchGeom mg = march_geom(h, w);
            const unsigned g = (unsigned)((int64_t)mg.nbx * mg.nbands);
            auto go = [&](auto kern) { kern<<<g, b, 0, st>>>(U, F, C, h, w, ld, out, partials, ticket); };
            const int sel = (bnd == BND_ZERO ? 4 : 0) | (f ? 2 : 0) | (clean ? 1 : 0);
            switch (sel) {
                case 0: go(energy_march_kernel<BND_REPLICATE, false, false>); break;
                case 1: go(energy_march_kernel<BND_REPLICATE, false, true>); break;
                case 2: go(energy_march_kernel<BND_REPLICATE, true, false>); break;
                case 3: go(energy_march_kernel<BND_REPLICATE, true, true>); break;
                case 4: go(energy_march_kernel<BND_ZERO, false, false>); break;
                case 5: go(energy_march_kernel<BND_ZERO, false, true>); break;
                case 6: go(energy_march_kernel<BND_ZERO, true, false>); break;
                default: go(energy_march_kernel<BND_ZERO, true, true>); break;
            }
            return cudaGetLastError();
        }
    }
    const unsigned g = (unsigned)energy_grid(h, w);
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
