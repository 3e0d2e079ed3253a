// wmc_adjoint.cu -- reverse mode of the unrolled WMC flow and of the WMC energy.
//
// The paper minimises with H^w as a (negative) gradient and leaves the gradient of its own
// regulariser R_{H^w} for future work (Sec. III, after Eq. wmcr); these kernels supply the
// derivatives needed to train through the flow.  H^w is piecewise linear in U: at a pixel p
// whose selection (Eq. act) picked d_m, H^w(U)(p) = sum_o h_m(o) U(p + o), so on that piece
//   dH^w(p)/dU(q) = sum over taps o of h_m(o) with (p + o read as q),
// where REPLICATE folds taps that fall outside the image onto the clamped pixel and ZERO drops
// them.  The adjoint of one flow step U' = (1-step) U + step f + step lambda H^w(U) is then
//   g = (1-step) g' + step lambda sum_p g'(p) dH^w(p)/dU          ("gather": pass B)
//   dloss/dlambda += step sum_p g'(p) H^w(U)(p)                    (pass A)
//   dloss/df      += step g'   (and + g^0 at the end, since U^0 = f)
// with the selection held at its forward value (a subgradient where it switches).  Pass A
// recomputes H^w(U^t) with exactly the forward's FP32 operations, so it lands on the same piece,
// and records the kernel index m(p) in one byte per pixel.
#include "wmc_device.cuh"
#include "wmc_internal.h"
#include "wmc_stream.cuh"

namespace wmc {

// 12 * h_1 .. 12 * h_8 of Sec. IV-B as correlation taps, row-major from the top-left.
__constant__ float kH12Taps[8][9] = {
    {2, 2, 0, 4, -12, 0, 2, 2, 0},    // h1: west half window
    {2, 4, 2, 2, -12, 2, 0, 0, 0},    // h2: north
    {0, 2, 2, 0, -12, 4, 0, 2, 2},    // h3: east
    {0, 0, 0, 2, -12, 2, 2, 4, 2},    // h4: south
    {2, 4, 1, 4, -12, 0, 1, 0, 0},    // h5: north-west
    {1, 4, 2, 0, -12, 4, 0, 0, 1},    // h6: north-east
    {0, 0, 1, 0, -12, 4, 1, 4, 2},    // h7: south-east
    {1, 0, 0, 4, -12, 0, 2, 4, 1},    // h8: south-west
};

// select12 with the index (0..7 for h1..h8) of the candidate it returns: the same comparisons
// in the same order, so the same value and the same piece as the forward kernels.
__device__ __forceinline__ float select12_idx(float L, float a1, float a2, float a5, float a6,
                                              int *m) {
    const float aL = fabsf(L);
    // aj and jd track the winner's odd part and the kernel index of its "L + a_j" candidate
    // (h1, h2, h5, h6)
    float t = aL - fabsf(a1), aj = a1;
    int jd = 0;
    const float t2 = aL - fabsf(a2), t5 = aL - fabsf(a5), t6 = aL - fabsf(a6);
    if (fabsf(t2) < fabsf(t)) { t = t2; aj = a2; jd = 1; }
    if (fabsf(t5) < fabsf(t)) { t = t5; aj = a5; jd = 4; }
    if (fabsf(t6) < fabsf(t)) { t = t6; aj = a6; jd = 5; }
    const float Ls = fmaf(0x1p-40f, a1, L);
    // the value returned is L - sign(Ls)|a_j|: the "L + a_j" kernel when the signs of Ls and a_j
    // differ (or a_j = 0), else its antipode (index + 2: h3, h4, h7, h8)
    const bool use_direct = (aj == 0.0f) || (signbit(Ls) != signbit(aj));
    *m = use_direct ? jd : jd + 2;
    return __int_as_float(__float_as_int(t) ^ (__float_as_int(Ls) & 0x80000000));
}

// 12 H^w and the selected kernel index at the centre of a 3x3 neighbourhood (the forward's terms).
__device__ __forceinline__ float half_laplace12_sel(float nw, float n, float ne, float w, float c,
                                                    float e, float sw, float s, float se, int *m) {
    const Terms1 t = half_laplace12_terms(nw, n, ne, w, c, e, sw, s, se);
    return select12_idx(t.L, t.a1, t.a2, t.a5, t.a6, m);
}

// The same for two cells at once (lane .x, lane .y): the forward's packed terms.
__device__ __forceinline__ float2 half_laplace12_sel_x2(float2 nw, float2 n, float2 ne, float2 w,
                                                        float2 c, float2 e, float2 sw, float2 s,
                                                        float2 se, int *m0, int *m1) {
    const Terms2 t = half_laplace12_terms_x2(nw, n, ne, w, c, e, sw, s, se);
    return make_float2(select12_idx(t.L.x, t.a1.x, t.a2.x, t.a5.x, t.a6.x, m0),
                       select12_idx(t.L.y, t.a1.y, t.a2.y, t.a5.y, t.a6.y, m1));
}

__device__ __forceinline__ double warp_sum_d(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// ------------------------------------------------------------------------- one adjoint step
// One CTA owns a kTX x kTY tile of q and stages in shared memory
//   U on the tile + 2 rings (the selection of every p next to the tile needs U around p),
//   g on the tile + 1 ring (0 outside the image), and m(p) on the tile + 1 ring.
// Phase 1 loads (a warp per row, lanes along it; every load issued before the first store),
// phase 2 selects m(p) (and, for the flow, adds g(p) * 12 H^w(p) over the tile's own pixels into
// the dlambda partial; for the energy, sets g(p) = sign(H^w(p))), phase 3 gathers
//   g_out(q) = c_self g(q) + c_nb * sum_p sum_o [p + o reads q] W12[m(p)][o] g(p)
// with c_nb = step * lambda[img] / 12 (flow) or 1/12 (energy), and
//   grad_f(q) = (first ? 0 : grad_f(q)) + step g(q) (+ g_out(q) when last).
// In phases 2 and 3 a thread owns one column and walks kRows rows down it with a 3-row window in
// registers, so each new row costs 3 shared loads instead of 9.
constexpr int kTX = 64, kTY = 32, kAdjThreads = 256;
constexpr int kGroups = kAdjThreads / kTX;  // row groups
constexpr int kRows = kTY / kGroups;        // rows per thread

int64_t adjoint_blocks(int32_t h, int32_t w) {
    return (int64_t)((w + kTX - 1) / kTX) * ((h + kTY - 1) / kTY);
}

// The selection byte stores the kernel index times the byte size of a tap row, so that a tap is
// one shared load at [index + constant] with no address arithmetic.
constexpr int kTapRowBytes = 9 * sizeof(float);

__device__ __forceinline__ float tap_at(const float (&taps)[8][9], int moff, int o) {
    return *reinterpret_cast<const float *>(reinterpret_cast<const char *>(&taps[0][0]) + moff + 4 * o);
}

using AdjU = float[kTY + 4][kTX + 4];
using AdjG = float[kTY + 2][kTX + 2];
using AdjM = uint8_t[kTY + 2][kTX + 2];

// Selection at p = tile (r, cc) from its 3x3 U window; returns g(p) * 12 H^w(p) for the dlambda
// partial when p is one of the tile's own pixels (flow), else 0.
template <int BND, bool ENERGY, bool CHECK>
__device__ __forceinline__ float adjoint_select_one(AdjU &us, AdjG &gs, AdjM &ms, int r, int cc,
                                                    int x0, int y0, int h, int w, float nw, float n,
                                                    float ne, float wv, float ce, float e, float sw,
                                                    float sv, float se) {
    if (CHECK) {
        const int y = y0 + r, x = x0 + cc;
        if (y < 0 || y >= h || x < 0 || x >= w) {
            ms[r + 1][cc + 1] = 0;
            if (ENERGY) gs[r + 1][cc + 1] = 0.0f;
            return 0.0f;
        }
    }
    int m;
    const float h12 = half_laplace12_sel(nw, n, ne, wv, ce, e, sw, sv, se, &m);
    ms[r + 1][cc + 1] = (uint8_t)(m * kTapRowBytes);
    if (ENERGY) {
        gs[r + 1][cc + 1] = h12 > 0.0f ? 1.0f : (h12 < 0.0f ? -1.0f : 0.0f);
        return 0.0f;
    }
    return (r >= 0 && r < kTY && cc >= 0 && cc < kTX) ? gs[r + 1][cc + 1] * h12 : 0.0f;
}

// Phase-2 selections of one thread: tile columns l and l + 32 (the two lanes of packed FP32x2
// arithmetic), kSelRows rows down from r0, a 3-row window of operand pairs in registers.
constexpr int kSelRows = kTY / (kAdjThreads / 32);  // rows per thread in phase 2

template <int BND, bool ENERGY, bool CHECK>
__device__ __forceinline__ float adjoint_select_rows2(AdjU &us, AdjG &gs, AdjM &ms, int l, int r0,
                                                      int x0, int y0, int h, int w) {
    float acc = 0.0f;
    // operand pairs: column cc of the tile is us column cc + 2; its west/east are cc + 1 / cc + 3
    auto row3 = [&](int ur, float2 &wv, float2 &cv, float2 &ev) {
        wv = make_float2(us[ur][l + 1], us[ur][l + 33]);
        cv = make_float2(us[ur][l + 2], us[ur][l + 34]);
        ev = make_float2(us[ur][l + 3], us[ur][l + 35]);
    };
    float2 aw, ac, ae, bw, bc, be;
    row3(r0 + 1, aw, ac, ae);
    row3(r0 + 2, bw, bc, be);
#pragma unroll
    for (int k = 0; k < kSelRows; ++k) {
        const int r = r0 + k;
        float2 dw, dc, de;
        row3(r + 3, dw, dc, de);
        int m0, m1;
        const float2 h12 = half_laplace12_sel_x2(aw, ac, ae, bw, bc, be, dw, dc, de, &m0, &m1);
        bool in0 = true, in1 = true;
        if (CHECK) {
            const int y = y0 + r;
            const bool rin = (y >= 0) & (y < h);
            in0 = rin & (x0 + l < w);
            in1 = rin & (x0 + l + 32 < w);
        }
        ms[r + 1][l + 1] = in0 ? (uint8_t)(m0 * kTapRowBytes) : 0;
        ms[r + 1][l + 33] = in1 ? (uint8_t)(m1 * kTapRowBytes) : 0;
        if (ENERGY) {
            gs[r + 1][l + 1] = in0 ? (h12.x > 0.0f ? 1.0f : (h12.x < 0.0f ? -1.0f : 0.0f)) : 0.0f;
            gs[r + 1][l + 33] = in1 ? (h12.y > 0.0f ? 1.0f : (h12.y < 0.0f ? -1.0f : 0.0f)) : 0.0f;
        } else {
            // outside the image g = 0, so those cells add nothing
            acc = fmaf(gs[r + 1][l + 1], h12.x, acc);
            acc = fmaf(gs[r + 1][l + 33], h12.y, acc);
        }
        aw = bw; ac = bc; ae = be;
        bw = dw; bc = dc; be = de;
    }
    return acc;
}

// Gather of kRows outputs q down column c from row r0 (see the kernel's comment).
template <int BND, bool CHECK>
__device__ __forceinline__ void adjoint_gather_rows(AdjG &gs, AdjM &ms, float (&taps)[8][9],
                                                    float *__restrict__ g_out,
                                                    float *__restrict__ grad_f, int c, int r0,
                                                    int x0, int y0, int h, int w, int64_t ld,
                                                    float step, float c_self, float c_nb, int first,
                                                    int last) {
    const int qx = x0 + c;
    float g0[3], g1[3], g2[3];
    int m0[3], m1[3], m2[3];
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        g0[k] = gs[r0][c + k];
        m0[k] = ms[r0][c + k];
        g1[k] = gs[r0 + 1][c + k];
        m1[k] = ms[r0 + 1][c + k];
    }
    // the grad_f reads of all rows go out before the gather arithmetic
    float gfv[kRows];
#pragma unroll
    for (int j = 0; j < kRows; ++j) {
        gfv[j] = 0.0f;
        const int qy = y0 + r0 + j;
        if (grad_f && !first && (!CHECK || (qy < h && qx < w))) gfv[j] = grad_f[(int64_t)qy * ld + qx];
    }
    int64_t o = (int64_t)(y0 + r0) * ld + qx;
#pragma unroll
    for (int j = 0; j < kRows; ++j, o += ld) {
        const int r = r0 + j;
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            g2[k] = gs[r + 2][c + k];
            m2[k] = ms[r + 2][c + k];
        }
        const int qy = y0 + r;
        if (!CHECK || (qy < h && qx < w)) {
            // p = q + (dy, dx) reads q through its tap (-dy, -dx): index (1-dy)*3 + (1-dx);
            // p outside the image carries g = 0
            float a = 0.0f;
#pragma unroll
            for (int k = 0; k < 3; ++k) {
                a = fmaf(tap_at(taps, m0[k], 8 - k), g0[k], a);  // dy = -1
                a = fmaf(tap_at(taps, m1[k], 5 - k), g1[k], a);  // dy = 0
                a = fmaf(tap_at(taps, m2[k], 2 - k), g2[k], a);  // dy = +1
            }
            if (BND == BND_REPLICATE && CHECK) {
                // Taps that leave the image read the clamped pixel.  On the first row, the taps
                // of row-0 pixels pointing up (oy = -1) also read q; likewise for the last row,
                // the first and last columns, and, at a corner, the diagonal tap of q itself.
                const bool top = qy == 0, bottom = qy == h - 1, left = qx == 0, right = qx == w - 1;
#pragma unroll
                for (int k = 0; k < 3; ++k) {
                    if (top) a = fmaf(tap_at(taps, m1[k], 2 - k), g1[k], a);
                    if (bottom) a = fmaf(tap_at(taps, m1[k], 8 - k), g1[k], a);
                }
                if (left) {
                    a = fmaf(tap_at(taps, m0[1], 6), g0[1], a);
                    a = fmaf(tap_at(taps, m1[1], 3), g1[1], a);
                    a = fmaf(tap_at(taps, m2[1], 0), g2[1], a);
                }
                if (right) {
                    a = fmaf(tap_at(taps, m0[1], 8), g0[1], a);
                    a = fmaf(tap_at(taps, m1[1], 5), g1[1], a);
                    a = fmaf(tap_at(taps, m2[1], 2), g2[1], a);
                }
                if (top && left) a = fmaf(tap_at(taps, m1[1], 0), g1[1], a);
                if (top && right) a = fmaf(tap_at(taps, m1[1], 2), g1[1], a);
                if (bottom && left) a = fmaf(tap_at(taps, m1[1], 6), g1[1], a);
                if (bottom && right) a = fmaf(tap_at(taps, m1[1], 8), g1[1], a);
            }
            const float gq = g1[1];
            const float out = fmaf(c_nb, a, c_self * gq);
            g_out[o] = out;
            if (grad_f) {
                float v = fmaf(step, gq, gfv[j]);
                if (last) v += out;
                grad_f[o] = v;
            }
        }
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            g0[k] = g1[k]; m0[k] = m1[k];
            g1[k] = g2[k]; m1[k] = m2[k];
        }
    }
}

template <int BND, bool ENERGY>
__global__ void __launch_bounds__(kAdjThreads, 4)
    adjoint_step_kernel(const float *__restrict__ U, const float *__restrict__ g_in,
                        float *__restrict__ g_out, float *__restrict__ grad_f,
                        double *__restrict__ partials, const float *__restrict__ lam, float step,
                        float c_self, float c_nb_fixed, int first, int last, int h, int w, int64_t ld,
                        int64_t img_stride) {
    constexpr int UW = kTX + 4, UH = kTY + 4, GW = kTX + 2, GH = kTY + 2;
    constexpr int NW = kAdjThreads / 32;
    __shared__ float taps[8][9];
    __shared__ float us[UH][UW];
    __shared__ float gs[GH][GW];
    __shared__ uint8_t ms[GH][GW];
    __shared__ double red[NW];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    if (tid < 72) taps[tid / 9][tid % 9] = kH12Taps[tid / 9][tid % 9];
    const int64_t off = (int64_t)blockIdx.y * img_stride;
    U += off;
    g_out += off;
    if (!ENERGY) g_in += off;
    if (grad_f) grad_f += off;
    const int nbx = (w + kTX - 1) / kTX;
    const int by = (int)(blockIdx.x / nbx), bx = (int)(blockIdx.x - (unsigned)by * nbx);
    const int x0 = bx * kTX, y0 = by * kTY;

    // ---- phase 1: rows warp, warp + NW, ...; columns lane, lane + 32, lane + 64
    {
        constexpr int RU = (UH + NW - 1) / NW, RG = (GH + NW - 1) / NW;
        int ux[3], gx[3];
        bool uok[3], gok[3];
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            const int cu = lane + 32 * k, xu = x0 - 2 + cu;
            uok[k] = cu < UW && (BND == BND_REPLICATE || (xu >= 0 && xu < w));
            ux[k] = min(max(xu, 0), w - 1);
            const int cg = lane + 32 * k, xg = x0 - 1 + cg;
            gok[k] = cg < GW && xg >= 0 && xg < w;
            gx[k] = min(max(xg, 0), w - 1);
        }
        float uv[RU][3];
#pragma unroll
        for (int j = 0; j < RU; ++j) {
            const int r = warp + NW * j, y = y0 - 2 + r;
            const bool rok = r < UH && (BND == BND_REPLICATE || (y >= 0 && y < h));
            const float *row = U + (int64_t)min(max(y, 0), h - 1) * ld;
#pragma unroll
            for (int k = 0; k < 3; ++k) uv[j][k] = (rok && uok[k]) ? row[ux[k]] : 0.0f;
        }
        float gv[RG][3];
        if (!ENERGY) {
#pragma unroll
            for (int j = 0; j < RG; ++j) {
                const int r = warp + NW * j, y = y0 - 1 + r;
                const bool rok = r < GH && y >= 0 && y < h;
                const float *row = g_in + (int64_t)min(max(y, 0), h - 1) * ld;
#pragma unroll
                for (int k = 0; k < 3; ++k) gv[j][k] = (rok && gok[k]) ? row[gx[k]] : 0.0f;
            }
        }
#pragma unroll
        for (int j = 0; j < RU; ++j) {
            const int r = warp + NW * j;
#pragma unroll
            for (int k = 0; k < 3; ++k)
                if (r < UH && lane + 32 * k < UW) us[r][lane + 32 * k] = uv[j][k];
        }
        if (!ENERGY) {
#pragma unroll
            for (int j = 0; j < RG; ++j) {
                const int r = warp + NW * j;
#pragma unroll
                for (int k = 0; k < 3; ++k)
                    if (r < GH && lane + 32 * k < GW) gs[r][lane + 32 * k] = gv[j][k];
            }
        }
    }
    __syncthreads();

    // ---- phase 2: p at tile (r, c) <-> ms/gs[r + 1][c + 1], U window us[r + 1 .. r + 3][c + 1 .. c + 3]
    // Tiles whose ring lies inside the image (all but the border tiles) skip every bounds check.
    const bool interior = x0 >= 1 && y0 >= 1 && x0 + kTX < w && y0 + kTY < h;
    const int c = tid % kTX, grp = tid / kTX;
    float acc = 0.0f;
    if (interior)
        acc = adjoint_select_rows2<BND, ENERGY, false>(us, gs, ms, lane, warp * kSelRows, x0, y0, h, w);
    else
        acc = adjoint_select_rows2<BND, ENERGY, true>(us, gs, ms, lane, warp * kSelRows, x0, y0, h, w);
    // the ring: rows -1 and kTY (all kTX + 2 columns), columns -1 and kTX (rows 0 .. kTY-1)
    for (int i = tid; i < 2 * GW + 2 * kTY; i += kAdjThreads) {
        int r, cc;
        if (i < 2 * GW) {
            r = i < GW ? -1 : kTY;
            cc = (i < GW ? i : i - GW) - 1;
        } else {
            const int k = i - 2 * GW;
            cc = k < kTY ? -1 : kTX;
            r = k < kTY ? k : k - kTY;
        }
        adjoint_select_one<BND, ENERGY, true>(us, gs, ms, r, cc, x0, y0, h, w,
                                              us[r + 1][cc + 1], us[r + 1][cc + 2], us[r + 1][cc + 3],
                                              us[r + 2][cc + 1], us[r + 2][cc + 2], us[r + 2][cc + 3],
                                              us[r + 3][cc + 1], us[r + 3][cc + 2], us[r + 3][cc + 3]);
    }
    if (!ENERGY && partials) {
        const double sacc = warp_sum_d((double)acc);
        if (lane == 0) red[warp] = sacc;
    }
    __syncthreads();
    if (!ENERGY && partials && tid == 0) {
        double t = 0.0;
        for (int k = 0; k < NW; ++k) t += red[k];
        partials[(int64_t)blockIdx.y * gridDim.x + blockIdx.x] = t;
    }

    // ---- phase 3
    const float c_nb = ENERGY ? c_nb_fixed : step * __ldg(lam + blockIdx.y) / 12.0f;
    if (interior)
        adjoint_gather_rows<BND, false>(gs, ms, taps, g_out, grad_f, c, grp * kRows, x0, y0, h, w, ld,
                                        step, c_self, c_nb, first, last);
    else
        adjoint_gather_rows<BND, true>(gs, ms, taps, g_out, grad_f, c, grp * kRows, x0, y0, h, w, ld,
                                       step, c_self, c_nb, first, last);
}

// ---------------------------------------------------------------------------------- dlambda
// grad_lambda[i] = step / 12 * sum over steps t and CTAs b of partials[t][i][b], in a fixed order.
__global__ void lambda_grad_kernel(const double *__restrict__ partials, int K, int n, int nb,
                                   float step, float *__restrict__ grad_lambda) {
    const int img = blockIdx.x;
    const int64_t total = (int64_t)K * nb;
    // thread i adds the partials i, i + blockDim.x, ... of this image (t-major), then a fixed tree
    double a = 0.0;
    for (int64_t i = threadIdx.x; i < total; i += blockDim.x) {
        const int64_t t = i / nb, b = i - t * nb;
        a += partials[(t * n + img) * nb + b];
    }
    __shared__ double red[32];
    a = warp_sum_d(a);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = a;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int k = 0; k < (int)(blockDim.x + 31) / 32; ++k) t += red[k];
        grad_lambda[img] = (float)((double)step / 12.0 * t);
    }
}

// ------------------------------------------------------------------------------- launchers
cudaError_t launch_adjoint_step(int bnd, const float *U, const float *g_in, float *g_out,
                                float *grad_f, double *partials, const float *lam, float step,
                                int first, int last, int32_t n, int32_t h, int32_t w, int64_t ld,
                                int64_t img_stride, cudaStream_t st) {
    const int64_t nb = adjoint_blocks(h, w);
    if (nb > 0x7fffffffLL || n > 65535) return cudaErrorInvalidConfiguration;
    dim3 grid((unsigned)nb, (unsigned)n);
    const float c_self = 1.0f - step;
    if (bnd == BND_ZERO)
        adjoint_step_kernel<BND_ZERO, false><<<grid, kAdjThreads, 0, st>>>(U, g_in, g_out, grad_f, partials, lam, step, c_self, 0.0f, first, last, h, w, ld, img_stride);
    else
        adjoint_step_kernel<BND_REPLICATE, false><<<grid, kAdjThreads, 0, st>>>(U, g_in, g_out, grad_f, partials, lam, step, c_self, 0.0f, first, last, h, w, ld, img_stride);
    return cudaGetLastError();
}

cudaError_t launch_energy_grad(int bnd, const float *U, float *grad, int32_t h, int32_t w, int64_t ld,
                               cudaStream_t st) {
    const int64_t nb = adjoint_blocks(h, w);
    if (nb > 0x7fffffffLL) return cudaErrorInvalidConfiguration;
    dim3 grid((unsigned)nb, 1u);
    if (bnd == BND_ZERO)
        adjoint_step_kernel<BND_ZERO, true><<<grid, kAdjThreads, 0, st>>>(U, nullptr, grad, nullptr, nullptr, nullptr, 0.0f, 0.0f, 1.0f / 12.0f, 0, 0, h, w, ld, 0);
    else
        adjoint_step_kernel<BND_REPLICATE, true><<<grid, kAdjThreads, 0, st>>>(U, nullptr, grad, nullptr, nullptr, nullptr, 0.0f, 0.0f, 1.0f / 12.0f, 0, 0, h, w, ld, 0);
    return cudaGetLastError();
}

cudaError_t launch_lambda_grad(const double *partials, int32_t K, int32_t n, int64_t nb, float step,
                               float *grad_lambda, cudaStream_t st) {
    if (n <= 0) return cudaSuccess;
    lambda_grad_kernel<<<n, 256, 0, st>>>(partials, K, n, (int)nb, step, grad_lambda);
    return cudaGetLastError();
}

cudaError_t launch_stack_step(int bnd, const float *u, const float *f, float *out, const float *lam,
                              float step, int32_t n, int32_t h, int32_t w, int64_t ld,
                              int64_t img_stride, bool vec, cudaStream_t st) {
    StreamParams p{};
    p.u = u;
    p.f = f;
    p.out = out;
    p.ldu = p.ldf = p.ldo = ld;
    p.h = h;
    p.w = w;
    p.c_keep = 1.0f - step;
    p.c_f = step;
    p.img_stride = img_stride;
    p.lam = lam;
    p.step = step;
    if (n > 65535) return cudaErrorInvalidConfiguration;
    if (quad_aligned<float>(p) && img_stride % 4 == 0) {
        if (bnd == BND_ZERO) return launch_stream4<BND_ZERO, MODE_FLOW, true>(p, (unsigned)n, st);
        return launch_stream4<BND_REPLICATE, MODE_FLOW, true>(p, (unsigned)n, st);
    }
    const int64_t nb = (int64_t)((w + kStreamWarps * 64 - 1) / (kStreamWarps * 64)) *
                       ((h + kStreamRY - 1) / kStreamRY);
    if (nb > 0x7fffffffLL) return cudaErrorInvalidConfiguration;
    dim3 grid((unsigned)nb, (unsigned)n);
    const unsigned b = kStreamWarps * 32;
    if (bnd == BND_ZERO) {
        if (vec) stream_kernel<float, BND_ZERO, MODE_FLOW, true, true><<<grid, b, 0, st>>>(p);
        else stream_kernel<float, BND_ZERO, MODE_FLOW, false, true><<<grid, b, 0, st>>>(p);
    } else {
        if (vec) stream_kernel<float, BND_REPLICATE, MODE_FLOW, true, true><<<grid, b, 0, st>>>(p);
        else stream_kernel<float, BND_REPLICATE, MODE_FLOW, false, true><<<grid, b, 0, st>>>(p);
    }
    return cudaGetLastError();
}

}  // namespace wmc
