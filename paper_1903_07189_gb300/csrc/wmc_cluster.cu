// wmc_cluster.cu -- the whole WMC flow (Sec. V-B, Eq. MCF) of a small image in ONE launch: one
// thread-block cluster whose CTAs keep the image in their shared memory for all the iterations.
//
// A small image (PR1: 256 x 256) is bound by latency, not by bytes or arithmetic: a launch per few
// Jacobi steps covers it with a handful of CTAs, so most of the time goes to each launch's load
// and the serial steps of one CTA.  Here a cluster of C <= 16 CTAs (one per SM) splits the image
// into bands of kCRows rows; CTA r keeps rows [kCRows r, kCRows (r + 1)) plus one halo row above
// and below in two ping-pong buffers in shared memory, and f's term in registers.  Every step it
// computes its band from one buffer into the other; the threads that compute a band's first and
// last rows also store those values into the neighbouring CTAs' halo rows, through distributed
// shared memory, and one cluster barrier per step (release / acquire) makes them visible before
// the next step reads them.  The arithmetic is the tile kernel's (the packed pair stencil of
// half_laplace12_x2, the same update and storage rounding), so the result is the same bits.
//
// Image boundary.  ZERO: the ring of cells just outside the image starts at 0 and is never
// written.  REPLICATE: a cell on the image's edge also writes its new value into the ring cells
// that replicate it (the row above or below, the column left or right, the corner), in its own
// CTA or, for a band's halo row, in the neighbour's; cells outside the image are never written.
//
// Threads: 16 warps as 4 column groups x 4 row groups; lane l of warp (wc, wr) updates columns
// 64 wc + l and 64 wc + l + 32 (the two lanes of the packed FP32x2 arithmetic) of band rows
// 4 wr .. 4 wr + 3.  Images up to 256 x 256.
//
// Control flow is the same in every CTA of the cluster (no early return before the last barrier,
// no data-dependent wait), so every CTA reaches every barrier; no CTA leaves while another may
// still write into its shared memory (the barrier after the last step orders those writes).
#include <atomic>
#include <type_traits>

#include "wmc_window.cuh"

namespace wmc {

constexpr int kCWarpCols = 4;                             // 4 warps side by side: 256 columns
constexpr int kCCols = 64 * kCWarpCols;                   // 256 columns per band
constexpr int kCRows = 16;                                // rows per band
constexpr int kCMaxCtas = 16;
constexpr int kCPitch = kCCols + 4;   // shared pitch: image column x at index x + 1; -1 and w inside
constexpr int kCBuf = (kCRows + 2) * kCPitch;  // floats per buffer (band + 2 halo rows)
constexpr int kCWarpRows = 4;                             // warp rows: 16 warps, 4 rows per thread
constexpr int kCThreads = 32 * kCWarpCols * kCWarpRows;   // 512

struct ClusterParams {
    const void *u0;   // U^0 (device, pitch ld)
    const void *f;    // f or nullptr (mean-curvature flow)
    void *out;        // U^iters (pitch ldo)
    unsigned int *status;  // the call's status word, cleared (no wait here can run out)
    int64_t ld, ldo;
    int32_t h, w, iters;
    float c_keep, c_f, c_h;
};

__device__ __forceinline__ uint32_t cluster_rank() {
    uint32_t r;
    asm volatile("mov.u32 %0, %%cluster_ctarank;" : "=r"(r));
    return r;
}

// Address of the same shared-memory location in CTA `rank` of the cluster.
__device__ __forceinline__ uint32_t map_rank(uint32_t local, uint32_t rank) {
    uint32_t remote;
    asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(remote) : "r"(local), "r"(rank));
    return remote;
}

__device__ __forceinline__ void st_cluster(uint32_t addr, float v) {
    asm volatile("st.shared::cluster.f32 [%0], %1;" ::"r"(addr), "f"(v) : "memory");
}

__device__ __forceinline__ void cluster_arrive() {
    asm volatile("barrier.cluster.arrive.release.aligned;" ::: "memory");
}
// Arrival that orders none of the thread's earlier memory accesses (for threads that wrote
// nothing another CTA reads).
__device__ __forceinline__ void cluster_arrive_relaxed() {
    asm volatile("barrier.cluster.arrive.relaxed.aligned;" ::: "memory");
}
__device__ __forceinline__ void cluster_wait() {
    asm volatile("barrier.cluster.wait.acquire.aligned;" ::: "memory");
}
__device__ __forceinline__ void cluster_sync() {
    cluster_arrive();
    cluster_wait();
}

template <typename S, int BND, int WR = kCWarpRows>
__global__ void __launch_bounds__(32 * kCWarpCols * WR, 1) flow_cluster_kernel(const ClusterParams p) {
    constexpr int NT = 32 * kCWarpCols * WR;  // threads
    constexpr int RPT = kCRows / WR;          // rows per thread
    static_assert(kCRows % WR == 0 && RPT >= 2, "band rows split evenly, two or more per thread");
    extern __shared__ __align__(16) float smem[];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int rank = (int)cluster_rank(), nranks = (int)gridDim.x;
    const int h = p.h, w = p.w;
    const int y_band = kCRows * rank;  // image row of band row 0

    // ---- initial state: band rows -1 .. kCRows of U^0 (the boundary rule outside the image) in
    // buffer 0; the ring columns -1 and w in both buffers (they hold the rule's values throughout
    // for ZERO, and REPLICATE rewrites them every step)
    if (rank == 0 && tid == 0 && p.status) *p.status = 0u;
    for (int idx = tid; idx < 2 * kCBuf; idx += NT) smem[idx] = 0.0f;
    __syncthreads();
    for (int idx = tid; idx < (kCRows + 2) * (w + 2); idx += NT) {
        const int i = idx / (w + 2), j = idx - i * (w + 2);  // band row i - 1, image column j - 1
        const int y = y_band + i - 1, x = j - 1;
        float v = 0.0f;
        if (BND == BND_REPLICATE) {
            const int yc = min(max(y, 0), h - 1), xc = min(max(x, 0), w - 1);
            if (y >= -1 && y <= h) v = Store<S>::load(static_cast<const S *>(p.u0) + (int64_t)yc * p.ld + xc);
        } else if (y >= 0 && y < h && x >= 0 && x < w) {
            v = Store<S>::load(static_cast<const S *>(p.u0) + (int64_t)y * p.ld + x);
        }
        smem[i * kCPitch + j] = v;
    }

    // ---- per-thread geometry and f's term (registers, for the whole run)
    const int wc = warp % kCWarpCols, wr = warp / kCWarpCols;
    const int x0 = 64 * wc + lane, x1 = x0 + 32;  // image columns of the two cells
    const int j = x0 + 1;                         // shared column of the first cell
    const int ib = 1 + RPT * wr;                  // shared row of the first row
    const bool cin0 = x0 < w, cin1 = x1 < w;
    const bool first_rows = wr == 0, last_rows = wr == WR - 1;  // hold the band's edge rows
    // Warps whose rows are all inside the image and neither a band edge row nor the image's top
    // or bottom row take a lean path: no halo stores, no row checks, only the column mirror of
    // REPLICATE (the lanes of image columns 0 and w - 1).  The condition is the same for the
    // whole warp.  A one-column image, whose cells have ring cells on both sides, takes the full
    // path.
    const bool lean = !first_rows && !last_rows && y_band + ib - 1 + RPT - 1 < h - 1 && w > 1;
    // REPLICATE column mirror: a lane of image column 0 or w - 1 also writes the ring cell beside
    // it; m0 / m1 are the offsets of the two cells' mirror stores (a cell with no ring cell beside
    // it gets its own offset: the store rewrites the value just stored).  Only the warps holding
    // column 0 or w - 1 issue them.
    const int m0 = x0 == 0 ? -1 : (x0 == w - 1 ? 1 : 0);
    const int m1 = x1 == w - 1 ? 33 : 32;
    const bool mirror_warp = BND == BND_REPLICATE && ((wc == 0) | ((w - 1) / 64 == wc));
    float2 g[RPT];
    const float2 cf = make_float2(p.c_f, p.c_f);
#pragma unroll
    for (int k = 0; k < RPT; ++k) {
        const int y = y_band + ib - 1 + k;
        float a = 0.0f, b = 0.0f;
        if (p.f != nullptr && y < h) {
            const S *fr = static_cast<const S *>(p.f) + (int64_t)y * p.ld;
            if (cin0) a = Store<S>::load(fr + x0);
            if (cin1) b = Store<S>::load(fr + x1);
        }
        g[k] = __fmul2_rn(cf, make_float2(a, b));
    }
    const float2 ch = make_float2(p.c_h, p.c_h), ck = make_float2(p.c_keep, p.c_keep);
    const uint32_t up = (uint32_t)(rank - 1), down = (uint32_t)(rank + 1);
    // A value stored into a neighbour's halo row, with the ring cells that replicate it there
    // (REPLICATE: image columns -1 and w of that row; a halo row is never image row -1 or h).
    auto halo_store = [&](uint32_t a, float vx, float vy) {
        if (cin0) {
            st_cluster(a, vx);
            if (BND == BND_REPLICATE && x0 == 0) st_cluster(a - 4, vx);
            if (BND == BND_REPLICATE && x0 == w - 1) st_cluster(a + 4, vx);
        }
        if (cin1) {
            st_cluster(a + 128, vy);
            if (BND == BND_REPLICATE && x1 == w - 1) st_cluster(a + 132, vy);
        }
    };
    // Row k of this thread's rows: the update of its two cells from rows k - 1, k, k + 1 of
    // `src`, stored into `dst` (and into the neighbour's halo row for a band edge row, and into
    // the ring cells that replicate an image edge cell).
    auto row_out = [&](float *dst, int k, const Row3 &r0, const Row3 &r1, const Row3 &r2) {
        const float2 hw = half_laplace12_x2(r0.w, r0.c, r0.e, r1.w, r1.c, r1.e, r2.w, r2.c, r2.e);
        const float2 v = Store<S>::round2(__ffma2_rn(ch, hw, __ffma2_rn(ck, r1.c, g[k])));
        const int i = ib + k, y = y_band + i - 1;  // shared row, image row
        if (y >= h) return;
        float *d = dst + i * kCPitch + j;
        if (cin0) d[0] = v.x;
        if (cin1) d[32] = v.y;
        if (i == 1 && rank > 0)
            halo_store(map_rank((uint32_t)__cvta_generic_to_shared(dst + (kCRows + 1) * kCPitch + j), up), v.x, v.y);
        if (i == kCRows && rank + 1 < nranks)
            halo_store(map_rank((uint32_t)__cvta_generic_to_shared(dst + j), down), v.x, v.y);
        if (BND == BND_REPLICATE) {
            // the ring cells that replicate this cell: columns -1 / w, rows -1 / h (image rows -1
            // and h lie in this band or its halo rows), and the corners
            const bool top = y == 0, bottom = y == h - 1;
            auto mirror = [&](int x, float val, int jj) {
                if (x == 0) d[jj - 1] = val;
                if (x == w - 1) d[jj + 1] = val;
                if (top) {
                    d[jj - kCPitch] = val;
                    if (x == 0) d[jj - kCPitch - 1] = val;
                    if (x == w - 1) d[jj - kCPitch + 1] = val;
                }
                if (bottom) {
                    d[jj + kCPitch] = val;
                    if (x == 0) d[jj + kCPitch - 1] = val;
                    if (x == w - 1) d[jj + kCPitch + 1] = val;
                }
            };
            if (cin0) mirror(x0, v.x, 0);
            if (cin1) mirror(x1, v.y, 32);
        }
    };
    // A row that is neither a band edge row nor the image's bottom row, and inside the image
    // (no halo store, no row mirror; only the column mirror of REPLICATE).
    auto row_plain = [&](auto mirror, float *dst, int k, const Row3 &r0, const Row3 &r1, const Row3 &r2) {
        const float2 hw = half_laplace12_x2(r0.w, r0.c, r0.e, r1.w, r1.c, r1.e, r2.w, r2.c, r2.e);
        const float2 v = Store<S>::round2(__ffma2_rn(ch, hw, __ffma2_rn(ck, r1.c, g[k])));
        float *d = dst + (ib + k) * kCPitch + j;
        if (cin0) d[0] = v.x;
        if (cin1) d[32] = v.y;
        if constexpr (decltype(mirror)::value) {
            if (cin0) d[m0] = v.x;
            if (cin1) d[m1] = v.y;
        }
    };
    using Mirror = std::integral_constant<bool, BND == BND_REPLICATE>;
    using NoMirror = std::integral_constant<bool, false>;
    // bit k: row k of this thread's rows is plain (the same for the whole warp)
    uint32_t plain_rows = 0;
#pragma unroll
    for (int k = 0; k < RPT; ++k) {
        const int i = ib + k, y = y_band + i - 1;
        if (i != 1 && i != kCRows && y < h - 1 && w > 1) plain_rows |= 1u << k;
    }
    auto row_pick = [&](float *dst, int k, const Row3 &r0, const Row3 &r1, const Row3 &r2) {
        if ((plain_rows >> k) & 1u)
            row_plain(Mirror{}, dst, k, r0, r1, r2);
        else
            row_out(dst, k, r0, r1, r2);
    };
    // Every CTA of the cluster has started and filled its buffers before any CTA writes into
    // another's shared memory.
    cluster_sync();

    // ---- the iterations.  Each step first computes the band's two edge rows (the only ones
    // that read the halo rows, and the ones the neighbours need), stores them, and arrives at the
    // cluster barrier with release semantics; the other warps arrive at once (relaxed: they wrote
    // nothing another CTA reads), and the rest of the band is computed while the barrier
    // completes.  A CTA barrier then orders this CTA's own writes, and the cluster wait (acquire)
    // the neighbours' halo rows.  No CTA writes a neighbour's halo rows of step s + 1 before
    // every CTA has arrived at step s, i.e. before their readers (the edge rows of step s) are
    // done.
    for (int s = 0; s < p.iters; ++s) {
        const float *src = smem + (s & 1) * kCBuf;
        float *dst = smem + ((s + 1) & 1) * kCBuf;
        const float *rp = src + (ib - 1) * kCPitch + j;
        Row3 r0 = load_row3(rp), r1 = load_row3(rp + kCPitch), r2 = load_row3(rp + 2 * kCPitch);
        if (lean) {
            cluster_arrive_relaxed();
            auto rows = [&](auto mirror) {
#pragma unroll
                for (int k = 0; k < RPT; ++k) {
                    if (k > 0) {
                        r0 = r1;
                        r1 = r2;
                        r2 = load_row3(rp + (k + 2) * kCPitch);
                    }
                    row_plain(mirror, dst, k, r0, r1, r2);
                }
            };
            if (mirror_warp)
                rows(Mirror{});
            else
                rows(NoMirror{});
        } else {
            if (first_rows) row_out(dst, 0, r0, r1, r2);
            if (last_rows)
                row_out(dst, RPT - 1, load_row3(rp + (RPT - 1) * kCPitch), load_row3(rp + RPT * kCPitch),
                        load_row3(rp + (RPT + 1) * kCPitch));
            cluster_arrive();
            if (!first_rows) row_pick(dst, 0, r0, r1, r2);
#pragma unroll
            for (int k = 1; k < RPT; ++k) {
                r0 = r1;
                r1 = r2;
                r2 = load_row3(rp + (k + 2) * kCPitch);
                if (k < RPT - 1 || !last_rows) row_pick(dst, k, r0, r1, r2);
            }
        }
        __syncthreads();
        cluster_wait();
    }

    // ---- U^iters: the band's own rows
    const float *fin = smem + (p.iters & 1) * kCBuf;
    for (int idx = tid; idx < kCRows * w; idx += NT) {
        const int i = idx / w, x = idx - i * w, y = y_band + i;
        if (y < h) Store<S>::store(static_cast<S *>(p.out) + (int64_t)y * p.ldo + x, fin[(i + 1) * kCPitch + x + 1]);
    }
}

// Cluster size for an h x w image, 0 if this path does not apply (larger than one cluster holds).
int cluster_ctas(int32_t h, int32_t w) {
    if (h < 1 || w < 1 || w > kCCols || h > kCRows * kCMaxCtas) return 0;
    return (h + kCRows - 1) / kCRows;
}

template <typename S, int BND>
static cudaError_t launch_cluster_t(const ClusterParams &p, int ctas, cudaStream_t st) {
    auto kern = flow_cluster_kernel<S, BND>;
    const size_t smem = 2 * kCBuf * sizeof(float);
    static std::atomic<uint64_t> attr_set{0};
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    const uint64_t bit = 1ull << (dev & 63);
    if (!(attr_set.load(std::memory_order_acquire) & bit)) {
        e = cudaFuncSetAttribute(kern, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
        if (e == cudaSuccess) e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
        attr_set.fetch_or(bit, std::memory_order_release);
    }
    cudaLaunchConfig_t cfg{};
    cfg.gridDim = dim3((unsigned)ctas);
    cfg.blockDim = dim3(kCThreads);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = (unsigned)ctas;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, kern, p);
}

// Whether a cluster of `ctas` CTAs of the kernel can be scheduled on the current device (asked
// once per device and size; any failure of the query reads as "no").
bool cluster_fits(int ctas) {
    if (ctas < 1 || ctas > kCMaxCtas) return false;
    static std::atomic<uint32_t> asked[64], fits[64];  // per device: one bit per cluster size
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    const uint32_t bit = 1u << (ctas - 1);
    if (asked[dev & 63].load(std::memory_order_acquire) & bit)
        return (fits[dev & 63].load(std::memory_order_acquire) & bit) != 0;
    auto kern = flow_cluster_kernel<float, BND_REPLICATE>;
    const size_t smem = 2 * kCBuf * sizeof(float);
    bool ok = cudaFuncSetAttribute(kern, cudaFuncAttributeNonPortableClusterSizeAllowed, 1) == cudaSuccess &&
              cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) == cudaSuccess;
    if (ok) {
        cudaLaunchConfig_t cfg{};
        cfg.gridDim = dim3((unsigned)ctas);
        cfg.blockDim = dim3(kCThreads);
        cfg.dynamicSmemBytes = smem;
        cudaLaunchAttribute attr[1];
        attr[0].id = cudaLaunchAttributeClusterDimension;
        attr[0].val.clusterDim.x = (unsigned)ctas;
        attr[0].val.clusterDim.y = 1;
        attr[0].val.clusterDim.z = 1;
        cfg.attrs = attr;
        cfg.numAttrs = 1;
        int n = 0;
        ok = cudaOccupancyMaxActiveClusters(&n, kern, &cfg) == cudaSuccess && n >= 1;
    }
    cudaGetLastError();
    if (ok) fits[dev & 63].fetch_or(bit, std::memory_order_acq_rel);
    asked[dev & 63].fetch_or(bit, std::memory_order_acq_rel);
    return ok;
}

cudaError_t launch_flow_cluster(int dtype, int bnd, const void *u0, const void *f, void *out,
                                unsigned int *status, int64_t ld, int64_t ldo, int32_t h, int32_t w,
                                int32_t iters, float c_keep, float c_f, float c_h, cudaStream_t st) {
    const int ctas = cluster_ctas(h, w);
    if (ctas == 0) return cudaErrorInvalidValue;
    ClusterParams p{u0, f, out, status, ld, ldo, h, w, iters, c_keep, c_f, c_h};
    const bool z = bnd == BND_ZERO;
    switch (dtype) {
        case 0: return z ? launch_cluster_t<float, BND_ZERO>(p, ctas, st) : launch_cluster_t<float, BND_REPLICATE>(p, ctas, st);
        case 1: return z ? launch_cluster_t<__nv_bfloat16, BND_ZERO>(p, ctas, st)
                         : launch_cluster_t<__nv_bfloat16, BND_REPLICATE>(p, ctas, st);
        case 2: return z ? launch_cluster_t<__half, BND_ZERO>(p, ctas, st) : launch_cluster_t<__half, BND_REPLICATE>(p, ctas, st);
        default: return cudaErrorInvalidValue;
    }
}

}  // namespace wmc
