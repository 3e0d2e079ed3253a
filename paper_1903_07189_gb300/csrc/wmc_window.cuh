// wmc_window.cuh -- pieces shared by the kernels that stage image windows in shared memory (the
// persistent evaluation and energy kernels and the temporally blocked flow kernel): the natural
// window geometry of a 128 x 64 box, TMA / mbarrier / programmatic-launch helpers with bounded
// waits, the REPLICATE ring refresh, and the packed row reads of the (j, j + 32) lane layout.
#pragma once

#include <cuda.h>
#include <string.h>

#include <algorithm>
#include <atomic>

#include "wmc_device.cuh"
#include "wmc_internal.h"

namespace wmc {

constexpr int kCW = 128;   // box columns
constexpr int kCH = 64;    // box rows
constexpr int kRY = 8;     // rows per thread in the (j, j + 32) lane layout
constexpr int kTileWX = 2; // warps across (64 columns each)
constexpr int kTileWY = kCH / kRY;  // warps down
constexpr int kTileThreadsV2 = 32 * kTileWX * kTileWY;  // 512

// Natural window of a box: the box's 128 columns start 2 + d (d < A) into the window, which
// starts on a 16-byte boundary (A elements), plus one halo cell on each side.
template <typename S> struct Geom {
    static constexpr int A = 16 / (int)sizeof(S);                 // TMA x alignment (elements)
    static constexpr int LW = ((kCW + 2 + A + A - 1) / A) * A;    // loaded width
    static constexpr int LH = kCH + 2;                            // loaded height
    static constexpr int P = LW;                                  // shared pitch (elements)
    static constexpr int BUF = LH * P;                            // elements per window
};

// Programmatic dependent launch: a launch made with the programmatic-serialization attribute may
// start while the previous kernel in the stream finishes (its CTAs fill the SMs the last wave
// leaves idle and do their set-up); griddep_wait() then blocks until that kernel has completed
// and its writes are visible.  Both are no-ops for a launch made without the attribute.
__device__ __forceinline__ void griddep_launch_dependents() {
    asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
}
__device__ __forceinline__ void griddep_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }

// Per-tile completion flags in global memory (a release store by the writing CTA; relaxed loads
// and a fence by the reader).
__device__ __forceinline__ unsigned int ld_relaxed_gpu(const unsigned int *p) {
    unsigned int v;
    asm volatile("ld.relaxed.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}
__device__ __forceinline__ void st_release_gpu(unsigned int *p, unsigned int v) {
    asm volatile("st.release.gpu.global.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}
// Orders this thread's earlier global-memory view of the generic proxy (including what its
// acquire loads made visible) before its later async-proxy (TMA) reads of global memory.
__device__ __forceinline__ void fence_proxy_async_global() {
    asm volatile("fence.proxy.async.global;" ::: "memory");
}

// ------------------------------------------------------------------ TMA / mbarrier helpers
__device__ __forceinline__ uint32_t smem_u32(const void *p) {
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ uint64_t global_timer_ns() {
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

__device__ __forceinline__ void mbar_init(uint32_t bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

__device__ __forceinline__ void mbar_arrive(uint32_t bar) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(bar) : "memory");
}

__device__ __forceinline__ void mbar_expect_tx(uint32_t bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes)
                 : "memory");
}

// Orders this thread's (and, after a CTA barrier, the CTA's) earlier shared-memory accesses of
// the generic proxy before later async-proxy (TMA) accesses of the same memory: issued before a
// TMA copy refills a buffer that threads have been reading.
__device__ __forceinline__ void fence_proxy_async_smem() {
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

__device__ __forceinline__ void tma_load_2d(uint32_t dst, const CUtensorMap *map, int x, int y,
                                            uint32_t bar) {
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.tile.mbarrier::complete_tx::bytes"
        " [%0], [%1, {%2, %3}], [%4];" ::"r"(dst),
        "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(bar)
        : "memory");
}

// Wait for the barrier's phase; give up after `limit_ns` (returns false).  Each try_wait may
// suspend the thread in hardware for up to 1 ms, so the loop spins very little.
__device__ __forceinline__ bool mbar_wait_bounded(uint32_t bar, uint32_t phase, uint64_t limit_ns) {
    const uint64_t t0 = global_timer_ns();
    for (;;) {
        uint32_t done;
        asm volatile(
            "{ .reg .pred p; mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2, %3;"
            " selp.u32 %0, 1, 0, p; }"
            : "=r"(done)
            : "r"(bar), "r"(phase), "r"(1000000u)
            : "memory");
        if (done) return true;
        if (global_timer_ns() - t0 > limit_ns) return false;
    }
}

constexpr uint64_t kWaitLimitNs = 200ull * 1000 * 1000;  // 0.2 s

// Columns j-1, j, j+1 of one shared row for both lanes (j and j+32) as aligned pairs.
struct Row3 {
    float2 w, c, e;
};
__device__ __forceinline__ Row3 load_row3(const float *r) {
    Row3 o;
    o.w = make_float2(r[-1], r[31]);
    o.c = make_float2(r[0], r[32]);
    o.e = make_float2(r[1], r[33]);
    return o;
}

// REPLICATE: set the ring of cells just outside the image (image rows -1 and h, image columns -1
// and w, where they cross the window) to the value of the nearest in-image cell, so that in-image
// cells can read their neighbours without clamping.  Corner cells belong to two segments and get
// the same value from both.
// The window is LW = Geom<S>::LW columns (pitch LW) by LH rows, and NT threads share the work.
template <typename S, int LH = Geom<S>::LH, int NT = kTileThreadsV2>
__device__ __forceinline__ void refresh_ring(float *buf, int X0, int Y0, int h, int w, int tid) {
    using G = Geom<S>;
    constexpr int LW = G::LW, P = G::P;
    const int ir0 = -1 - Y0, ir1 = h - Y0;  // shared rows of image rows -1 and h
    const int jc0 = -1 - X0, jc1 = w - X0;  // shared columns of image columns -1 and w
    const int jlo = max(jc0, 0), jhi = min(jc1, LW - 1);
    const int ilo = max(ir0, 0), ihi = min(ir1, LH - 1);
    for (int t = tid; t < 2 * (LW + LH); t += NT) {
        int i, j2;
        if (t < 2 * LW) {
            i = (t < LW) ? ir0 : ir1;
            j2 = (t < LW) ? t : t - LW;
            if (i < 0 || i >= LH || j2 < jlo || j2 > jhi) continue;
        } else {
            const int q = t - 2 * LW;
            j2 = (q < LH) ? jc0 : jc1;
            i = (q < LH) ? q : q - LH;
            if (j2 < 0 || j2 >= LW || i < ilo || i > ihi) continue;
        }
        const int yy = Y0 + i, xx = X0 + j2;
        const int ci = min(max(yy, 0), h - 1) - Y0, cj = min(max(xx, 0), w - 1) - X0;
        buf[i * P + j2] = buf[ci * P + cj];
    }
}


}  // namespace wmc
