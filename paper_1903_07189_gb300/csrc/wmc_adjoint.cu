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

// half_laplace12 with the index (0..7 for h1..h8) of the candidate it returns.  Same FP32
// operations, hence the same value and the same piece as the forward kernels.
__device__ __forceinline__ float half_laplace12_sel(float nw, float n, float ne, float w, float c,
                                                    float e, float sw, float s, float se, int *m) {
    const float p = n - s;
    const float q = w - e;
    const float A = nw - se;
    const float B = ne - sw;
    const float corners = (nw + se) + (ne + sw);
    const float edges = (n + s) + (w + e);
    const float L = fmaf(-12.0f, c, fmaf(2.0f, edges, corners));
    const float a[4] = {fmaf(2.0f, q, A - B), fmaf(2.0f, p, A + B), fmaf(2.0f, p + q, A),
                        fmaf(2.0f, p - q, B)};
    const float aL = fabsf(L);
    float t = aL - fabsf(a[0]);
    int j = 0;
#pragma unroll
    for (int k = 1; k < 4; ++k) {
        const float tk = aL - fabsf(a[k]);
        if (fabsf(tk) < fabsf(t)) {
            t = tk;
            j = k;
        }
    }
    const float Ls = fmaf(0x1p-40f, a[0], L);
    // candidate L + a_j is h_{direct}, L - a_j its antipode; the value returned is
    // L - sign(Ls)|a_j|, i.e. + a_j exactly when the signs of Ls and a_j differ
    const int direct[4] = {0, 1, 4, 5}, anti[4] = {2, 3, 6, 7};
    const bool use_direct = (a[j] == 0.0f) || (signbit(Ls) != signbit(a[j]));
    *m = use_direct ? direct[j] : anti[j];
    return __int_as_float(__float_as_int(t) ^ (__float_as_int(Ls) & 0x80000000));
}

__device__ __forceinline__ double warp_sum_d(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// ---------------------------------------------------------------------------------- pass A
// For every pixel p of image blockIdx.y: m(p) and either
//   - partials[blockIdx.y * gridDim.x + blockIdx.x] = sum over the CTA's pixels of g(p) * 12 H^w(p)
//   - or, when sign_out != nullptr, sign_out(p) = sign(H^w(p)) (energy gradient).
template <int BND>
__global__ void __launch_bounds__(kStreamWarps * 32)
    adjoint_select_kernel(const float *__restrict__ U, const float *__restrict__ g,
                          uint8_t *__restrict__ mout, float *__restrict__ sign_out,
                          double *__restrict__ partials, int h, int w, int64_t ld,
                          int64_t img_stride) {
    constexpr int R = kStreamRY;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int nbx = (w + kStreamWarps * 64 - 1) / (kStreamWarps * 64);
    const int by = (int)(blockIdx.x / nbx), bx = (int)(blockIdx.x - (unsigned)by * nbx);
    const int x = ((bx * kStreamWarps + warp) * 32 + lane) * 2;
    const int y0 = by * R;
    const int64_t off = (int64_t)blockIdx.y * img_stride;
    U += off;
    mout += off;
    if (g) g += off;
    if (sign_out) sign_out += off;
    float acc = 0.0f;
    if ((x & ~63) < w) {
        float2 v[R + 2];
        float el[R + 2], er[R + 2];
#pragma unroll
        for (int k = 0; k < R + 2; ++k) {
            bool ok;
            const int y = row_index<BND>(y0 - 1 + k, h, &ok);
            const float *row = U + (int64_t)y * ld;
            v[k] = load_pair<float, BND, false>(row, x, w, ok);
            el[k] = (lane == 0) ? load_one<float, BND>(row, x - 1, w, ok) : 0.0f;
            er[k] = (lane == 31) ? load_one<float, BND>(row, x + 2, w, ok) : 0.0f;
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
            int m0, m1;
            const float h0 = half_laplace12_sel(lf[k], v[k].x, v[k].y, lf[k + 1], v[k + 1].x,
                                                v[k + 1].y, lf[k + 2], v[k + 2].x, v[k + 2].y, &m0);
            const float h1 = half_laplace12_sel(v[k].x, v[k].y, rt[k], v[k + 1].x, v[k + 1].y,
                                                rt[k + 1], v[k + 2].x, v[k + 2].y, rt[k + 2], &m1);
            const int64_t o = (int64_t)y * ld + x;
            if (x < w) {
                mout[o] = (uint8_t)m0;
                if (sign_out) sign_out[o] = h0 > 0.0f ? 1.0f : (h0 < 0.0f ? -1.0f : 0.0f);
                if (g) acc = fmaf(g[o], h0, acc);
            }
            if (x + 1 < w) {
                mout[o + 1] = (uint8_t)m1;
                if (sign_out) sign_out[o + 1] = h1 > 0.0f ? 1.0f : (h1 < 0.0f ? -1.0f : 0.0f);
                if (g) acc = fmaf(g[o + 1], h1, acc);
            }
        }
    }
    if (!partials) return;
    __shared__ double red[kStreamWarps];
    const double s = warp_sum_d((double)acc);
    if (lane == 0) red[warp] = s;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int i = 0; i < kStreamWarps; ++i) t += red[i];
        partials[(int64_t)blockIdx.y * gridDim.x + blockIdx.x] = t;
    }
}

// ---------------------------------------------------------------------------------- pass B
// g_out(q) = c_self * g_in(q) + c_nb(img) * sum_p sum_o [p + o reads q] W12[m(p)][o] g_in(p)
// with c_nb = step * lambda[img] / 12 (flow) or 1/12 (energy), and optionally
//   grad_f(q) = (first ? 0 : grad_f(q)) + step * g_in(q) (+ g_out(q) when last).
constexpr int kGX = 32, kGY = 8;

template <int BND>
__global__ void __launch_bounds__(kGX * kGY)
    adjoint_gather_kernel(const float *__restrict__ g_in, const uint8_t *__restrict__ m,
                          float *__restrict__ g_out, float *__restrict__ grad_f,
                          const float *__restrict__ lam, float step, float c_self, float c_nb_fixed,
                          int first, int last, int h, int w, int64_t ld, int64_t img_stride) {
    __shared__ float taps[8][9];
    __shared__ float gs[kGY + 2][kGX + 2];
    __shared__ uint8_t ms[kGY + 2][kGX + 2];
    const int tid = threadIdx.y * kGX + threadIdx.x;
    if (tid < 72) taps[tid / 9][tid % 9] = kH12Taps[tid / 9][tid % 9];
    const int64_t off = (int64_t)blockIdx.z * img_stride;
    g_in += off;
    m += off;
    g_out += off;
    if (grad_f) grad_f += off;
    const int qx0 = blockIdx.x * kGX, qy0 = blockIdx.y * kGY;
    // halo tile: g and m of p = q + (-1..1, -1..1); pixels outside the image carry g = 0
    for (int i = tid; i < (kGY + 2) * (kGX + 2); i += kGX * kGY) {
        const int r = i / (kGX + 2), c = i % (kGX + 2);
        const int y = qy0 - 1 + r, x = qx0 - 1 + c;
        const bool in = (y >= 0) & (y < h) & (x >= 0) & (x < w);
        gs[r][c] = in ? g_in[(int64_t)y * ld + x] : 0.0f;
        ms[r][c] = in ? m[(int64_t)y * ld + x] : 0;
    }
    __syncthreads();
    const int qx = qx0 + threadIdx.x, qy = qy0 + threadIdx.y;
    if (qx >= w || qy >= h) return;
    const float c_nb = lam ? step * __ldg(lam + blockIdx.z) / 12.0f : c_nb_fixed;
    float acc = 0.0f;
    const bool edge = (BND == BND_REPLICATE) &&
                      ((qx == 0) | (qx == w - 1) | (qy == 0) | (qy == h - 1));
    if (!edge) {
        // every p = q - o inside the image read q through tap o only
#pragma unroll
        for (int dy = -1; dy <= 1; ++dy)
#pragma unroll
            for (int dx = -1; dx <= 1; ++dx) {
                const int r = threadIdx.y + 1 + dy, c = threadIdx.x + 1 + dx;
                const int o = (1 - dy) * 3 + (1 - dx);  // tap of p that reads q
                acc = fmaf(taps[ms[r][c]][o], gs[r][c], acc);
            }
    } else {
        // image edge under REPLICATE: p's taps that fall outside the image read the clamped
        // pixel, so several taps of one p may read q
        for (int dy = -1; dy <= 1; ++dy)
            for (int dx = -1; dx <= 1; ++dx) {
                const int py = qy + dy, px = qx + dx;
                if (py < 0 || py >= h || px < 0 || px >= w) continue;
                const int r = threadIdx.y + 1 + dy, c = threadIdx.x + 1 + dx;
                const float gp = gs[r][c];
                const int mm = ms[r][c];
                for (int oy = -1; oy <= 1; ++oy)
                    for (int ox = -1; ox <= 1; ++ox) {
                        const int ry = min(max(py + oy, 0), h - 1), rx = min(max(px + ox, 0), w - 1);
                        if (ry == qy && rx == qx) acc = fmaf(taps[mm][(oy + 1) * 3 + (ox + 1)], gp, acc);
                    }
            }
    }
    const float gq = gs[threadIdx.y + 1][threadIdx.x + 1];
    const float out = fmaf(c_nb, acc, c_self * gq);
    const int64_t o = (int64_t)qy * ld + qx;
    g_out[o] = out;
    if (grad_f) {
        float v = first ? 0.0f : grad_f[o];
        v = fmaf(step, gq, v);
        if (last) v += out;
        grad_f[o] = v;
    }
}

// ---------------------------------------------------------------------------------- dlambda
// grad_lambda[i] = step / 12 * sum over steps t and CTAs b of partials[t][i][b], in a fixed order.
__global__ void lambda_grad_kernel(const double *__restrict__ partials, int K, int n, int nb,
                                   float step, float *__restrict__ grad_lambda) {
    const int i = blockIdx.x;
    double a = 0.0;
    for (int t = 0; t < K; ++t)
        for (int b = threadIdx.x; b < nb; b += blockDim.x)
            a += partials[((int64_t)t * n + i) * nb + b];
    __shared__ double red[32];
    a = warp_sum_d(a);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = a;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int k = 0; k < (int)(blockDim.x + 31) / 32; ++k) t += red[k];
        grad_lambda[i] = (float)((double)step / 12.0 * t);
    }
}

// ------------------------------------------------------------------------------- launchers
int64_t adjoint_select_blocks(int32_t h, int32_t w) {
    const int64_t nbx = (w + kStreamWarps * 64 - 1) / (kStreamWarps * 64);
    const int64_t nby = (h + kStreamRY - 1) / kStreamRY;
    return nbx * nby;
}

cudaError_t launch_adjoint_select(int bnd, const float *U, const float *g, uint8_t *m,
                                  float *sign_out, double *partials, int32_t n, int32_t h,
                                  int32_t w, int64_t ld, int64_t img_stride, cudaStream_t st) {
    const int64_t nb = adjoint_select_blocks(h, w);
    if (nb > 0x7fffffffLL || n > 65535) return cudaErrorInvalidConfiguration;
    dim3 grid((unsigned)nb, (unsigned)n);
    if (bnd == BND_ZERO)
        adjoint_select_kernel<BND_ZERO><<<grid, kStreamWarps * 32, 0, st>>>(U, g, m, sign_out, partials, h, w, ld, img_stride);
    else
        adjoint_select_kernel<BND_REPLICATE><<<grid, kStreamWarps * 32, 0, st>>>(U, g, m, sign_out, partials, h, w, ld, img_stride);
    return cudaGetLastError();
}

cudaError_t launch_adjoint_gather(int bnd, const float *g_in, const uint8_t *m, float *g_out,
                                  float *grad_f, const float *lam, float step, float c_self,
                                  float c_nb, int first, int last, int32_t n, int32_t h, int32_t w,
                                  int64_t ld, int64_t img_stride, cudaStream_t st) {
    if (n > 65535 || (h + kGY - 1) / kGY > 65535) return cudaErrorInvalidConfiguration;
    dim3 grid((unsigned)((w + kGX - 1) / kGX), (unsigned)((h + kGY - 1) / kGY), (unsigned)n);
    dim3 block(kGX, kGY);
    if (bnd == BND_ZERO)
        adjoint_gather_kernel<BND_ZERO><<<grid, block, 0, st>>>(g_in, m, g_out, grad_f, lam, step, c_self, c_nb, first, last, h, w, ld, img_stride);
    else
        adjoint_gather_kernel<BND_REPLICATE><<<grid, block, 0, st>>>(g_in, m, g_out, grad_f, lam, step, c_self, c_nb, first, last, h, w, ld, img_stride);
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
    const int64_t nb = adjoint_select_blocks(h, w);
    if (nb > 0x7fffffffLL || n > 65535) return cudaErrorInvalidConfiguration;
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
