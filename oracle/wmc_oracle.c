/*
 * wmc_oracle.c -- plain, slow FP64 CPU reference for the Weighted Mean Curvature (WMC)
 * "Half Laplace Operator" of Gong & Goksel, "Weighted Mean Curvature" (arXiv 1903.07189),
 * and for the WMC-regularised image updates built on it.
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the oracle the CUDA library is checked against.
 * Only the test-suite, the smoke check and the CPU-baseline leg of the benchmark load it.
 * It shares no code, header, table or helper with the CUDA path, and the CUDA path never
 * calls it.
 *
 * Everything is written the way the paper states it, with no blocking, fusion or
 * reordering:
 *   - the eight half-window kernels h_1..h_8 are the matrices printed in Sec. IV-B; they
 *     are stored as integer numerators over 12 (the Appendix writes its two base kernels the
 *     same way, as integer matrices divided by 6 and 12), so that integer-valued test
 *     images are evaluated exactly;
 *   - d_i = h_i * U for i = 1..8 (Eq. conv), applying each printed matrix as a correlation
 *     (entry (r,c) multiplies U[y+r-1][x+c-1], rows running downwards);
 *   - H^w = d_m with m = argmin_i |d_i| (Eq. act).  The paper does not say which candidate
 *     wins a tie; the Appendix listing takes the first minimum of its list, and its list,
 *     read as correlation kernels, is (h3, h1, h4, h2, h7, h8, h6, h5).  That order is used;
 *   - outside the image: REPLICATE (clamped index, the discrete Neumann rule of Sec. III-C and
 *     Sec. IV-A) or ZERO (the zero padding of the Appendix listing's conv2 'same');
 *   - the update U^{t+1} = U^t + step * (lambda * H^w(U^t) - mu * (U^t - f)) is the explicit
 *     gradient flow of Sec. V-B with A = I (mu = 1), and the mean-curvature flow of
 *     Eq. MCF when mu = 0; every pixel of step t reads U^t (Jacobi order);
 *   - the energies are the WMC regulariser of Eq. wmcr with q = 1 (sum |H^w|), the L2 data
 *     term of Eq. 1 (1/2 sum (U-f)^2) and the squared error to a clean image.
 *   - the L1-fidelity primal-dual update of Sec. V-C (shrinkage of r = U - f + d, clipping
 *     of the scaled dual d, then the U step with lambda H^w - (2 d^{t+1} - d^t)/alpha).
 *   - storage rounding: FP64 -> bfloat16 / binary16 round-to-nearest-even, taken straight from
 *     the FP64 bit pattern (no double rounding through FP32).
 *   - the conventional discretisation the paper compares against (Sec. V-D): Eq. rhs,
 *     H = Laplacian(U) - (U_y^2 U_yy + 2 U_x U_y U_xy + U_x^2 U_xx) / (U_x^2 + U_y^2), with
 *     central differences (unit spacing, rows downwards) and the same boundary rules.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define ORACLE_BND_REPLICATE 0
#define ORACLE_BND_ZERO 1

/* Rows of a whole-image pass may be split across OpenMP threads (every pixel is computed on
 * its own, so the result does not depend on the thread count).  Default: 1 thread. */
static int g_threads = 1;

void oracle_set_threads(int n) { g_threads = n > 0 ? n : 1; }
int oracle_get_threads(void) { return g_threads; }

/* 12 * h_i, i = 1..8, exactly as printed in Sec. IV-B (row r = 0 is the top row). */
static const int H12[8][3][3] = {
    /* h1 */ {{2, 2, 0}, {4, -12, 0}, {2, 2, 0}},
    /* h2 */ {{2, 4, 2}, {2, -12, 2}, {0, 0, 0}},
    /* h3 */ {{0, 2, 2}, {0, -12, 4}, {0, 2, 2}},
    /* h4 */ {{0, 0, 0}, {2, -12, 2}, {2, 4, 2}},
    /* h5 */ {{2, 4, 1}, {4, -12, 0}, {1, 0, 0}},
    /* h6 */ {{1, 4, 2}, {0, -12, 4}, {0, 0, 1}},
    /* h7 */ {{0, 0, 1}, {0, -12, 4}, {1, 4, 2}},
    /* h8 */ {{1, 0, 0}, {4, -12, 0}, {2, 4, 1}},
};

/* First-minimum order of the Appendix listing, as 0-based indices of h_1..h_8. */
static const int CANON[8] = {2, 0, 3, 1, 6, 7, 5, 4};

/* Expose the kernel table (as doubles) so tests can compare it with the printed matrices. */
void oracle_kernel(int i, double out[9]) {
    for (int r = 0; r < 3; ++r)
        for (int c = 0; c < 3; ++c) out[3 * r + c] = H12[i][r][c] / 12.0;
}

void oracle_canonical_order(int out[8]) {
    for (int k = 0; k < 8; ++k) out[k] = CANON[k];
}

/* U[y][x] with the boundary rule applied outside [0,h) x [0,w). */
static double sample(const double *u, int32_t h, int32_t w, int64_t ld, int32_t y, int32_t x,
                     int bnd) {
    if (y < 0 || y >= h || x < 0 || x >= w) {
        if (bnd == ORACLE_BND_ZERO) return 0.0;
        if (y < 0) y = 0;
        if (y >= h) y = h - 1;
        if (x < 0) x = 0;
        if (x >= w) x = w - 1;
    }
    return u[(int64_t)y * ld + x];
}

/* The eight signed distances d_1..d_8 at (y,x), Eq. conv (index i-1 holds d_i). */
static void distances(const double *u, int32_t h, int32_t w, int64_t ld, int32_t y, int32_t x,
                      int bnd, double d[8]) {
    for (int i = 0; i < 8; ++i) {
        double acc = 0.0;
        for (int r = 0; r < 3; ++r)
            for (int c = 0; c < 3; ++c)
                acc += (double)H12[i][r][c] * sample(u, h, w, ld, y + r - 1, x + c - 1, bnd);
        d[i] = acc / 12.0;
    }
}

/* Eq. act: first candidate of CANON with the smallest |d|; returns its 0-based kernel index. */
static int select_min(const double d[8]) {
    int m = CANON[0];
    for (int k = 1; k < 8; ++k) {
        int i = CANON[k];
        if (fabs(d[i]) < fabs(d[m])) m = i;
    }
    return m;
}

static int check_dims(int32_t h, int32_t w, int64_t ld) {
    if (h < 0 || w < 0) return 1;
    if (h > 0 && w > 0 && ld < w) return 1;
    return 0;
}

/*
 * H^w for every pixel.  hw: h x w with leading dimension ld_hw.
 * cand (optional, may be NULL): h*w*8 doubles, pixel-major, d_1..d_8 at each pixel.
 * index (optional): h*w bytes, the selected kernel index m in 1..8.
 * Returns 0, or 1 on bad sizes.
 */
int oracle_wmc_eval(const double *u, double *hw, int32_t h, int32_t w, int64_t ld_u,
                    int64_t ld_hw, int bnd, double *cand, uint8_t *index) {
    if (check_dims(h, w, ld_u) || (h > 0 && w > 0 && ld_hw < w)) return 1;
#pragma omp parallel for schedule(static) num_threads(g_threads)
    for (int32_t y = 0; y < h; ++y)
        for (int32_t x = 0; x < w; ++x) {
            double d[8];
            distances(u, h, w, ld_u, y, x, bnd, d);
            int m = select_min(d);
            hw[(int64_t)y * ld_hw + x] = d[m];
            if (cand)
                for (int i = 0; i < 8; ++i) cand[((int64_t)y * w + x) * 8 + i] = d[i];
            if (index) index[(int64_t)y * w + x] = (uint8_t)(m + 1);
        }
    return 0;
}

/* Round a double to the nearest bfloat16 (ties to even) and back, from the FP64 bits. */
static double round_bf16(double v) {
    if (isnan(v) || isinf(v) || v == 0.0) return v;
    /* bfloat16: 8 exponent bits (bias 127), 7 fraction bits; subnormals below 2^-126. */
    int e;
    frexp(v, &e); /* v = m * 2^e, 0.5 <= |m| < 1  => unit in last place = 2^(e-1-7) */
    int ulp_exp = e - 8;
    if (ulp_exp < -133) ulp_exp = -133; /* subnormal spacing 2^-133 */
    double scaled = ldexp(v, -ulp_exp);  /* exact: scaling by a power of two */
    double r = nearbyint(scaled);        /* round-half-even in the default mode */
    double out = ldexp(r, ulp_exp);
    if (fabs(out) > 3.3895313892515355e38) out = copysign(INFINITY, v);
    return out;
}

/* Round a double to the nearest IEEE binary16 (ties to even) and back. */
static double round_f16(double v) {
    if (isnan(v) || isinf(v) || v == 0.0) return v;
    int e;
    frexp(v, &e);
    int ulp_exp = e - 11; /* 10 fraction bits */
    if (ulp_exp < -24) ulp_exp = -24; /* subnormal spacing 2^-24 */
    double scaled = ldexp(v, -ulp_exp);
    double r = nearbyint(scaled);
    double out = ldexp(r, ulp_exp);
    if (fabs(out) >= 65520.0) out = copysign(INFINITY, v);
    return out;
}

/* storage: 0 = none (FP64), 1 = bfloat16, 2 = binary16, 3 = binary32. */
double oracle_round_storage(double v, int storage) {
    switch (storage) {
        case 1: return round_bf16(v);
        case 2: return round_f16(v);
        case 3: return (double)(float)v;
        default: return v;
    }
}

/*
 * Explicit WMC gradient flow, `iters` Jacobi steps starting from u0 (u0 == NULL: U^0 = f):
 *   U^{t+1} = U^t + step * (lambda * H^w(U^t) - mu * (U^t - f)).
 * mu = 1: L2 denoising with A = I (Sec. V-B); mu = 0: mean-curvature flow (Eq. MCF; f unused,
 * may be NULL when u0 is given).  storage != 0 rounds f, U^0 and every U^{t+1} to that storage
 * format, to mirror reduced-precision storage.  Dense h x w arrays with leading dimension ld.
 * Returns 0, 1 on bad arguments, 2 on allocation failure.
 */
int oracle_wmc_flow(const double *f, const double *u0, double *u_out, int32_t h, int32_t w,
                    int64_t ld, double lambda, double step, int32_t iters, int bnd, double mu,
                    int storage) {
    if (check_dims(h, w, ld) || iters < 0) return 1;
    if (!u0 && !f) return 1;
    if (mu != 0.0 && !f) return 1;
    if (h == 0 || w == 0) return 0;
    size_t n = (size_t)h * (size_t)w;
    double *U = (double *)malloc(n * sizeof(double));
    double *V = (double *)malloc(n * sizeof(double));
    double *F = (double *)malloc(n * sizeof(double));
    double *Hw = (double *)malloc(n * sizeof(double));
    if (!U || !V || !F || !Hw) {
        free(U); free(V); free(F); free(Hw);
        return 2;
    }
    const double *src = u0 ? u0 : f;
    for (int32_t y = 0; y < h; ++y)
        for (int32_t x = 0; x < w; ++x) {
            U[(size_t)y * w + x] = oracle_round_storage(src[(int64_t)y * ld + x], storage);
            F[(size_t)y * w + x] = f ? oracle_round_storage(f[(int64_t)y * ld + x], storage) : 0.0;
        }
    for (int32_t t = 0; t < iters; ++t) {
        oracle_wmc_eval(U, Hw, h, w, w, w, bnd, NULL, NULL);
#pragma omp parallel for schedule(static) num_threads(g_threads)
        for (size_t p = 0; p < n; ++p) {
            double next = U[p] + step * (lambda * Hw[p] - mu * (U[p] - F[p]));
            V[p] = oracle_round_storage(next, storage);
        }
        double *tmp = U; U = V; V = tmp;
    }
    for (int32_t y = 0; y < h; ++y)
        for (int32_t x = 0; x < w; ++x) u_out[(int64_t)y * ld + x] = U[(size_t)y * w + x];
    free(U); free(V); free(F); free(Hw);
    return 0;
}

/*
 * Energies (FP64): out[0] = sum |H^w(U)| (Eq. wmcr, q = 1); out[1] = 1/2 sum (U - f)^2 (the
 * L2 data term with A = I; 0 if f is NULL); out[2] = sum (U - clean)^2 (0 if clean is NULL).
 */
int oracle_energies(const double *u, const double *f, const double *clean, int32_t h,
                    int32_t w, int64_t ld, int bnd, double out[3]) {
    out[0] = out[1] = out[2] = 0.0;
    if (check_dims(h, w, ld)) return 1;
    for (int32_t y = 0; y < h; ++y)
        for (int32_t x = 0; x < w; ++x) {
            double d[8];
            distances(u, h, w, ld, y, x, bnd, d);
            int64_t p = (int64_t)y * ld + x;
            out[0] += fabs(d[select_min(d)]);
            if (f) out[1] += 0.5 * (u[p] - f[p]) * (u[p] - f[p]);
            if (clean) out[2] += (u[p] - clean[p]) * (u[p] - clean[p]);
        }
    return 0;
}

/*
 * L1-fidelity primal-dual iteration of Sec. V-C with A = I, from U^0 = u0 (or f) and d^0 = d0
 * (or 0):
 *   r = U^t - f + d^t;  d^{t+1} = clip(r, -alpha, alpha);
 *   U^{t+1} = U^t + step * (lambda * H^w(U^t) - (2 d^{t+1} - d^t) / alpha).
 * d_out (optional) receives d^iters.  Returns 0, 1 on bad arguments, 2 on allocation failure.
 */
int oracle_wmc_l1_primal_dual(const double *f, const double *u0, const double *d0, double *u_out,
                              double *d_out,
                              int32_t h, int32_t w, int64_t ld, double lambda, double step,
                              double alpha, int32_t iters, int bnd) {
    if (check_dims(h, w, ld) || iters < 0 || !f || !(alpha > 0.0)) return 1;
    if (h == 0 || w == 0) return 0;
    size_t n = (size_t)h * (size_t)w;
    double *U = (double *)malloc(n * sizeof(double));
    double *V = (double *)malloc(n * sizeof(double));
    double *D = (double *)calloc(n, sizeof(double));
    double *Hw = (double *)malloc(n * sizeof(double));
    if (!U || !V || !D || !Hw) {
        free(U); free(V); free(D); free(Hw);
        return 2;
    }
    const double *src = u0 ? u0 : f;
    for (int32_t y = 0; y < h; ++y)
        for (int32_t x = 0; x < w; ++x) {
            U[(size_t)y * w + x] = src[(int64_t)y * ld + x];
            if (d0) D[(size_t)y * w + x] = d0[(int64_t)y * ld + x];
        }
    for (int32_t t = 0; t < iters; ++t) {
        oracle_wmc_eval(U, Hw, h, w, w, w, bnd, NULL, NULL);
        for (int32_t y = 0; y < h; ++y)
            for (int32_t x = 0; x < w; ++x) {
                size_t p = (size_t)y * w + x;
                double r = U[p] - f[(int64_t)y * ld + x] + D[p];
                double dn = r > alpha ? alpha : (r < -alpha ? -alpha : r);
                V[p] = U[p] + step * (lambda * Hw[p] - (2.0 * dn - D[p]) / alpha);
                D[p] = dn;
            }
        double *tmp = U; U = V; V = tmp;
    }
    for (int32_t y = 0; y < h; ++y)
        for (int32_t x = 0; x < w; ++x) {
            u_out[(int64_t)y * ld + x] = U[(size_t)y * w + x];
            if (d_out) d_out[(int64_t)y * ld + x] = D[(size_t)y * w + x];
        }
    free(U); free(V); free(D); free(Hw);
    return 0;
}

/*
 * Opposite-sign near-ties of Eq. act, the events the parity protocol excuses: pixels where the
 * candidates d_i whose magnitude lies within `tau` of the smallest magnitude include both a
 * positive and a negative value (so two valid choices of d_m differ by about 2 |d_m|).  Counts
 * them over the whole image; returns 0, or 1 on bad arguments.
 */
int oracle_count_ties(const double *u, int32_t h, int32_t w, int64_t ld, int bnd, double tau,
                      int64_t *count) {
    if (check_dims(h, w, ld) || !(tau >= 0.0) || !count) return 1;
    int64_t n = 0;
#pragma omp parallel for schedule(static) num_threads(g_threads) reduction(+ : n)
    for (int32_t y = 0; y < h; ++y)
        for (int32_t x = 0; x < w; ++x) {
            double d[8];
            distances(u, h, w, ld, y, x, bnd, d);
            double mn = fabs(d[0]);
            for (int i = 1; i < 8; ++i)
                if (fabs(d[i]) < mn) mn = fabs(d[i]);
            int pos = 0, neg = 0;
            for (int i = 0; i < 8; ++i)
                if (fabs(d[i]) <= mn + tau) {
                    pos |= d[i] > 0.0;
                    neg |= d[i] < 0.0;
                }
            n += pos & neg;
        }
    *count = n;
    return 0;
}

/*
 * Point-sampled forms for checks at sizes where the whole-image oracle is too slow.
 * oracle_wmc_eval_points: H^w (Eq. conv + Eq. act) at n pixels (ys[k], xs[k]); cand (optional)
 * receives the eight d_i of each pixel (n*8 doubles).
 * oracle_wmc_step_points: one Jacobi step of the flow above at n pixels, given U^t and f
 * (f may be NULL when mu == 0); cand as above.
 */
int oracle_wmc_eval_points(const double *u, int32_t h, int32_t w, int64_t ld, int bnd,
                           const int32_t *ys, const int32_t *xs, int64_t n, double *out,
                           double *cand) {
    if (check_dims(h, w, ld)) return 1;
    for (int64_t k = 0; k < n; ++k) {
        if (ys[k] < 0 || ys[k] >= h || xs[k] < 0 || xs[k] >= w) return 1;
        double d[8];
        distances(u, h, w, ld, ys[k], xs[k], bnd, d);
        out[k] = d[select_min(d)];
        if (cand)
            for (int i = 0; i < 8; ++i) cand[k * 8 + i] = d[i];
    }
    return 0;
}

int oracle_wmc_step_points(const double *f, const double *u, int32_t h, int32_t w, int64_t ld,
                           double lambda, double step, double mu, int bnd, const int32_t *ys,
                           const int32_t *xs, int64_t n, double *out, double *cand) {
    if (check_dims(h, w, ld) || (mu != 0.0 && !f)) return 1;
    for (int64_t k = 0; k < n; ++k) {
        if (ys[k] < 0 || ys[k] >= h || xs[k] < 0 || xs[k] >= w) return 1;
        double d[8];
        distances(u, h, w, ld, ys[k], xs[k], bnd, d);
        int64_t p = (int64_t)ys[k] * ld + xs[k];
        double fp = f ? f[p] : 0.0;
        out[k] = u[p] + step * (lambda * d[select_min(d)] - mu * (u[p] - fp));
        if (cand)
            for (int i = 0; i < 8; ++i) cand[k * 8 + i] = d[i];
    }
    return 0;
}

/*
 * Unrolled L2 denoising and its gradient.  U^0 = f and, for t < K (Sec. V-B with A = I),
 *   U^{t+1} = U^t + step (lambda H^w(U^t) - (U^t - f));   loss = (1/N) sum_p (U^K(p) - clean(p))^2.
 * H^w is piecewise linear in U: where the selection m(p) of Eq. act is fixed, H^w(U)(p) is the
 * correlation of U with h_{m(p)} at p.  The gradient takes that piece (a subgradient where m
 * switches), i.e. the chain rule through each step with m(p) held at its forward value:
 *   g^K = dloss/dU^K = 2 (U^K - clean) / N
 *   g^t = (1 - step) g^{t+1} + step lambda sum_p g^{t+1}(p) dH^w(U^t)(p)/dU^t
 *   dloss/dlambda = step sum_t sum_p g^{t+1}(p) H^w(U^t)(p)
 *   dloss/df      = step sum_t g^{t+1} + g^0
 * where dH^w(p)/dU(q) is the weight of h_{m(p)} on the tap that reads q; under REPLICATE the
 * taps outside the image read the clamped pixel and carry their weight to it, under ZERO they
 * read nothing.  Dense h x w arrays (pitch w).  Returns 0, 1 on bad arguments, 2 on allocation
 * failure.
 */
int oracle_unrolled_grad(const double *f, const double *clean, int32_t h, int32_t w, double lambda,
                         double step, int32_t K, int bnd, double *loss, double *grad_lambda,
                         double *grad_f) {
    if (h <= 0 || w <= 0 || K < 0 || !f || !clean) return 1;
    const size_t n = (size_t)h * (size_t)w;
    double *U = (double *)malloc((size_t)(K + 1) * n * sizeof(double));
    double *Hs = (double *)malloc((size_t)(K > 0 ? K : 1) * n * sizeof(double));
    uint8_t *Ms = (uint8_t *)malloc((size_t)(K > 0 ? K : 1) * n);
    double *g = (double *)malloc(n * sizeof(double));
    double *gn = (double *)malloc(n * sizeof(double));
    if (!U || !Hs || !Ms || !g || !gn) {
        free(U); free(Hs); free(Ms); free(g); free(gn);
        return 2;
    }
    memcpy(U, f, n * sizeof(double));
    for (int32_t t = 0; t < K; ++t) {
        const double *Ut = U + (size_t)t * n;
        double *Un = U + (size_t)(t + 1) * n;
        for (int32_t y = 0; y < h; ++y)
            for (int32_t x = 0; x < w; ++x) {
                double d[8];
                distances(Ut, h, w, w, y, x, bnd, d);
                const int m = select_min(d);
                const size_t p = (size_t)y * w + x;
                Hs[(size_t)t * n + p] = d[m];
                Ms[(size_t)t * n + p] = (uint8_t)m;
                Un[p] = Ut[p] + step * (lambda * d[m] - (Ut[p] - f[p]));
            }
    }
    const double *UK = U + (size_t)K * n;
    double l = 0.0;
    for (size_t p = 0; p < n; ++p) {
        const double r = UK[p] - clean[p];
        l += r * r;
        g[p] = 2.0 * r / (double)n;
    }
    *loss = l / (double)n;
    double gl = 0.0;
    for (size_t p = 0; p < n; ++p) grad_f[p] = 0.0;
    for (int32_t t = K - 1; t >= 0; --t) {
        for (size_t p = 0; p < n; ++p) {
            gl += step * g[p] * Hs[(size_t)t * n + p];
            grad_f[p] += step * g[p];
            gn[p] = (1.0 - step) * g[p];
        }
        for (int32_t y = 0; y < h; ++y)
            for (int32_t x = 0; x < w; ++x) {
                const size_t p = (size_t)y * w + x;
                const int m = Ms[(size_t)t * n + p];
                for (int r = 0; r < 3; ++r)
                    for (int c = 0; c < 3; ++c) {
                        int qy = y + r - 1, qx = x + c - 1;
                        if (qy < 0 || qy >= h || qx < 0 || qx >= w) {
                            if (bnd == ORACLE_BND_ZERO) continue;
                            qy = qy < 0 ? 0 : (qy >= h ? h - 1 : qy);
                            qx = qx < 0 ? 0 : (qx >= w ? w - 1 : qx);
                        }
                        gn[(size_t)qy * w + qx] += step * lambda * (H12[m][r][c] / 12.0) * g[p];
                    }
            }
        double *tmp = g; g = gn; gn = tmp;
    }
    for (size_t p = 0; p < n; ++p) grad_f[p] += g[p];
    *grad_lambda = gl;
    free(U); free(Hs); free(Ms); free(g); free(gn);
    return 0;
}

/*
 * Gradient of the WMC regulariser E = sum_p |H^w(U)(p)| (Eq. wmcr, q = 1) with each pixel's
 * selection held fixed: dE/dU(q) = sum_p sign(H^w(p)) dH^w(p)/dU(q), the weight of h_{m(p)} on
 * the tap that reads q (folded onto the clamped pixel under REPLICATE, dropped under ZERO);
 * sign(0) = 0.  grad: dense h x w (pitch w).  Returns 0 or 1 on bad sizes.
 */
int oracle_energy_grad(const double *u, int32_t h, int32_t w, int bnd, double *grad) {
    if (h <= 0 || w <= 0 || !u || !grad) return 1;
    for (size_t p = 0; p < (size_t)h * w; ++p) grad[p] = 0.0;
    for (int32_t y = 0; y < h; ++y)
        for (int32_t x = 0; x < w; ++x) {
            double d[8];
            distances(u, h, w, w, y, x, bnd, d);
            const int m = select_min(d);
            const double s = d[m] > 0 ? 1.0 : (d[m] < 0 ? -1.0 : 0.0);
            for (int r = 0; r < 3; ++r)
                for (int c = 0; c < 3; ++c) {
                    int qy = y + r - 1, qx = x + c - 1;
                    if (qy < 0 || qy >= h || qx < 0 || qx >= w) {
                        if (bnd == ORACLE_BND_ZERO) continue;
                        qy = qy < 0 ? 0 : (qy >= h ? h - 1 : qy);
                        qx = qx < 0 ? 0 : (qx >= w ? w - 1 : qx);
                    }
                    grad[(size_t)qy * w + qx] += s * (H12[m][r][c] / 12.0);
                }
        }
    return 0;
}

/*
 * Conventional finite-difference WMC of Eq. rhs, the comparator of Sec. V-D: at every pixel
 *   U_x = (E - W)/2, U_y = (S - N)/2, U_xx = E - 2C + W, U_yy = S - 2C + N,
 *   U_xy = ((SE - NE) - (SW - NW))/4   (y runs downwards, so S is row y+1),
 *   H = (U_xx + U_yy) - (U_y^2 U_yy + 2 U_x U_y U_xy + U_x^2 U_xx) / (U_x^2 + U_y^2),
 * and H = 0 where the central-difference gradient is exactly zero (the |grad U| factor of
 * Eq. wmc vanishes there).  Neighbours outside the image follow `bnd`.
 */
int oracle_fd_eval(const double *u, double *hw, int32_t h, int32_t w, int64_t ld_u, int64_t ld_hw,
                   int bnd) {
    if (check_dims(h, w, ld_u) || check_dims(h, w, ld_hw)) return 1;
#pragma omp parallel for schedule(static) num_threads(g_threads)
    for (int32_t y = 0; y < h; ++y)
        for (int32_t x = 0; x < w; ++x) {
            const double C = sample(u, h, w, ld_u, y, x, bnd);
            const double N = sample(u, h, w, ld_u, y - 1, x, bnd);
            const double S = sample(u, h, w, ld_u, y + 1, x, bnd);
            const double W = sample(u, h, w, ld_u, y, x - 1, bnd);
            const double E = sample(u, h, w, ld_u, y, x + 1, bnd);
            const double NW = sample(u, h, w, ld_u, y - 1, x - 1, bnd);
            const double NE = sample(u, h, w, ld_u, y - 1, x + 1, bnd);
            const double SW = sample(u, h, w, ld_u, y + 1, x - 1, bnd);
            const double SE = sample(u, h, w, ld_u, y + 1, x + 1, bnd);
            const double ux = (E - W) / 2.0, uy = (S - N) / 2.0;
            const double uxx = E - 2.0 * C + W, uyy = S - 2.0 * C + N;
            const double uxy = ((SE - NE) - (SW - NW)) / 4.0;
            const double g2 = ux * ux + uy * uy;
            double H = 0.0;
            if (g2 > 0.0)
                H = (uxx + uyy) - (uy * uy * uyy + 2.0 * ux * uy * uxy + ux * ux * uxx) / g2;
            hw[(int64_t)y * ld_hw + x] = H;
        }
    return 0;
}

/* The flow of oracle_wmc_flow with the finite-difference H of oracle_fd_eval (FP64 storage). */
int oracle_fd_flow(const double *f, const double *u0, double *u_out, int32_t h, int32_t w,
                   int64_t ld, double lambda, double step, int32_t iters, int bnd, double mu) {
    if (check_dims(h, w, ld) || iters < 0) return 1;
    if (!u0 && !f) return 1;
    if (mu != 0.0 && !f) return 1;
    if (h == 0 || w == 0) return 0;
    size_t n = (size_t)h * (size_t)w;
    double *U = (double *)malloc(n * sizeof(double));
    double *V = (double *)malloc(n * sizeof(double));
    double *Hw = (double *)malloc(n * sizeof(double));
    if (!U || !V || !Hw) {
        free(U); free(V); free(Hw);
        return 2;
    }
    const double *src = u0 ? u0 : f;
    for (int32_t y = 0; y < h; ++y)
        for (int32_t x = 0; x < w; ++x) U[(size_t)y * w + x] = src[(int64_t)y * ld + x];
    for (int32_t t = 0; t < iters; ++t) {
        oracle_fd_eval(U, Hw, h, w, w, w, bnd);
        for (int32_t y = 0; y < h; ++y)
            for (int32_t x = 0; x < w; ++x) {
                const size_t p = (size_t)y * w + x;
                const double fv = f ? f[(int64_t)y * ld + x] : 0.0;
                V[p] = U[p] + step * (lambda * Hw[p] - mu * (U[p] - fv));
            }
        double *tmp = U; U = V; V = tmp;
    }
    for (int32_t y = 0; y < h; ++y)
        for (int32_t x = 0; x < w; ++x) u_out[(int64_t)y * ld + x] = U[(size_t)y * w + x];
    free(U); free(V); free(Hw);
    return 0;
}
