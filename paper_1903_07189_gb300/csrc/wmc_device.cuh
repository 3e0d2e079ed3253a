// wmc_device.cuh -- device-side arithmetic of the WMC Half Laplace Operator (sm_103a).
//
// H^w(U) = d_m, m = argmin_i |d_i|, d_i = h_i * U (Sec. IV-B, Eq. conv / Eq. act).
//
// The kernels here do not evaluate the eight 6-tap sums one by one.  The eight half windows
// come in antipodal pairs (h1,h3), (h2,h4), (h5,h7), (h6,h8) whose average is the isotropic
// Laplace kernel k4 of Eq. kernel3; so with L = k4 * U and the odd parts a_j = d_j - L
// (j = 1, 2, 5, 6) the candidates are exactly d = L +- a_j.  For one pair the smaller
// magnitude is ||L| - |a_j||, reached with the value sign(L) (|L| - |a_j|), so
//     H^w = sign(L) * t*,  t* = the t_j = |L| - |a_j| of smallest magnitude.
// In exact arithmetic this equals Eq. act (when L = 0 the two candidates of a pair are an
// opposite-sign tie and either is a valid d_m).  Everything is carried scaled by 12 so that
// all stencil weights are small integers:
//     12 L   = (NW + NE + SW + SE) + 2 (N + S + E + W) - 12 C
//     12 a_1 = (NW + SW - NE - SE) + 2 (W - E)          (h1: west half window)
//     12 a_2 = (NW + NE - SW - SE) + 2 (N - S)          (h2: north half window)
//     12 a_5 = (NW - SE) + 2 (N + W - S - E)            (h5: north-west half window)
//     12 a_6 = (NE - SW) + 2 (N + E - S - W)            (h6: north-east half window)
// which costs about 30 FP32 operations per pixel instead of ~60 for eight sums and eight
// compare/selects.
#pragma once

#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>
#include <stdint.h>

namespace wmc {

// Selection of Eq. act from the ×12 Laplacian L and odd parts a_j (j = 1, 2, 5, 6): the t_j =
// |L| - |a_j| of least magnitude, with the sign of L.  Ties between the t_j keep the first in
// the order 1, 2, 5, 6.  When L is exactly 0 the two candidates of every pair are an
// opposite-sign tie and RNE arithmetic gives L = +0 for U and for -U alike; taking the sign of
// L + 2^-40 a_1 instead makes the choice odd in U (H^w(-U) = -H^w(U) bit for bit) and changes
// nothing outside that tie band.
// Ls = L + 2^-40 a1 computed by the caller.
__device__ __forceinline__ float select12_ls(float L, float a1, float a2, float a5, float a6, float Ls) {
    const float aL = fabsf(L);
    float t = aL - fabsf(a1);
    const float t2 = aL - fabsf(a2);
    const float t5 = aL - fabsf(a5);
    const float t6 = aL - fabsf(a6);
    t = fabsf(t2) < fabsf(t) ? t2 : t;
    t = fabsf(t5) < fabsf(t) ? t5 : t;
    t = fabsf(t6) < fabsf(t) ? t6 : t;
    return __int_as_float(__float_as_int(t) ^ (__float_as_int(Ls) & 0x80000000));
}

__device__ __forceinline__ float select12(float L, float a1, float a2, float a5, float a6) {
    return select12_ls(L, a1, a2, a5, a6, fmaf(0x1p-40f, a1, L));
}


// The x12 Laplacian L and the odd parts a1, a2, a5, a6 at the centre of a 3x3 neighbourhood
// (rows: n* above, s* below), written through four values of each row so that a kernel walking
// down a column forms each row's once and shares them between the three cells that read that
// row.  For a row with cells (w, c, e):
//   P = w + 2c,  Q = 2c + e,  R = P + e,  D = w - e,
// and then, with q = D(centre),
//   L  = R(above) + R(below) + 2 R(centre) - 16 c   (= corners + 2 edges - 12 c)
//   a1 = 2 q + D(above) + D(below)                   (= 2 (w - e) + A - B)
//   a2 = R(above) - R(below)                         (= 2 (n - s) + A + B)
//   a5 = 2 q + P(above) - Q(below)                   (= 2 (p + q) + A)
//   a6 = -2 q + Q(above) - P(below)                  (= 2 (p - q) + B)
// with p = n - s, A = nw - se, B = ne - sw.  Every form of the stencil (scalar, packed, adjoint)
// takes these operations in this order, so they agree bit for bit.
struct Terms1 {
    float L, a1, a2, a5, a6;
};
__device__ __forceinline__ Terms1 half_laplace12_terms(float nw, float n, float ne, float w, float c,
                                                       float e, float sw, float s, float se) {
    const float Pa = fmaf(2.0f, n, nw), Qa = fmaf(2.0f, n, ne), Ra = Pa + ne, Da = nw - ne;
    const float Pc = fmaf(2.0f, c, w), Rc = Pc + e, q = w - e;
    const float Pb = fmaf(2.0f, s, sw), Qb = fmaf(2.0f, s, se), Rb = Pb + se, Db = sw - se;
    Terms1 t;
    t.L = fmaf(-16.0f, c, fmaf(2.0f, Rc, Ra + Rb));
    t.a1 = fmaf(2.0f, q, Da + Db);
    t.a2 = Ra - Rb;
    t.a5 = fmaf(2.0f, q, Pa - Qb);
    t.a6 = fmaf(-2.0f, q, Qa - Pb);
    return t;
}

// 12 * H^w at the centre of a 3x3 neighbourhood.
__device__ __forceinline__ float half_laplace12(float nw, float n, float ne, float w, float c,
                                                float e, float sw, float s, float se) {
    const Terms1 t = half_laplace12_terms(nw, n, ne, w, c, e, sw, s, se);
    return select12(t.L, t.a1, t.a2, t.a5, t.a6);
}

// Conventional finite-difference WMC of Eq. rhs at the centre of a 3x3 neighbourhood (rows: n*
// above, s* below), central differences with unit spacing:
//   H = (U_xx + U_yy) - (U_y^2 U_yy + 2 U_x U_y U_xy + U_x^2 U_xx) / (U_x^2 + U_y^2),
// and 0 where the central-difference gradient is exactly zero.  U_x and U_y are differences of
// two stored values (exact, or correct to one rounding), so the quotient keeps FP32 relative
// accuracy even where the gradient is small.
__device__ __forceinline__ float fd_wmc(float nw, float n, float ne, float w, float c, float e,
                                        float sw, float s, float se) {
    const float ux = 0.5f * (e - w), uy = 0.5f * (s - n);
    const float uxx = fmaf(-2.0f, c, e) + w, uyy = fmaf(-2.0f, c, s) + n;
    const float uxy = 0.25f * ((se - ne) - (sw - nw));
    const float g2 = fmaf(ux, ux, uy * uy);
    if (!(g2 > 0.0f)) return 0.0f;
    const float num = fmaf(uy * uy, uyy, fmaf(2.0f * ux * uy, uxy, ux * ux * uxx));
    return (uxx + uyy) - num / g2;
}

// The same for two cells at once (lane .x = one cell, .y = the other): the twenty linear
// operations run as packed FP32x2 instructions (sm_100+), each lane rounding exactly as the
// scalar operation above (a - b is computed as fma(b, -1, a), which is exact in the product),
// so both forms give bit-identical results.
__device__ __forceinline__ float2 sub2(float2 a, float2 b) {
    return __ffma2_rn(b, make_float2(-1.0f, -1.0f), a);
}
// The same linear part for two cells (the terms of half_laplace12_x2), operation for operation.
struct Terms2 {
    float2 L, a1, a2, a5, a6;
};
__device__ __forceinline__ Terms2 half_laplace12_terms_x2(float2 nw, float2 n, float2 ne, float2 w,
                                                          float2 c, float2 e, float2 sw, float2 s,
                                                          float2 se) {
    const float2 two = make_float2(2.0f, 2.0f), mtwo = make_float2(-2.0f, -2.0f);
    const float2 m16 = make_float2(-16.0f, -16.0f);
    const float2 Pa = __ffma2_rn(two, n, nw), Qa = __ffma2_rn(two, n, ne), Ra = __fadd2_rn(Pa, ne), Da = sub2(nw, ne);
    const float2 Pc = __ffma2_rn(two, c, w), Rc = __fadd2_rn(Pc, e), q = sub2(w, e);
    const float2 Pb = __ffma2_rn(two, s, sw), Qb = __ffma2_rn(two, s, se), Rb = __fadd2_rn(Pb, se), Db = sub2(sw, se);
    Terms2 t;
    t.L = __ffma2_rn(m16, c, __ffma2_rn(two, Rc, __fadd2_rn(Ra, Rb)));
    t.a1 = __ffma2_rn(two, q, __fadd2_rn(Da, Db));
    t.a2 = sub2(Ra, Rb);
    t.a5 = __ffma2_rn(two, q, sub2(Pa, Qb));
    t.a6 = __ffma2_rn(mtwo, q, sub2(Qa, Pb));
    return t;
}

// 12 |H^w| of two cells (the energies): the least |t_j| per lane, without the compare-select chain
// and the sign (equal magnitudes are equal values, so this is |half_laplace12_x2| bit for bit); the
// four differences |L| - |a_j| as packed adds, with the same roundings.
__device__ __forceinline__ float2 abs_half_laplace12_x2(float2 nw, float2 n, float2 ne, float2 w,
                                                        float2 c, float2 e, float2 sw, float2 s,
                                                        float2 se) {
    const Terms2 t = half_laplace12_terms_x2(nw, n, ne, w, c, e, sw, s, se);
    const float2 aL = make_float2(fabsf(t.L.x), fabsf(t.L.y));
    auto nabs = [](float2 v) { return make_float2(-fabsf(v.x), -fabsf(v.y)); };
    const float2 t1 = __fadd2_rn(aL, nabs(t.a1)), t2 = __fadd2_rn(aL, nabs(t.a2));
    const float2 t5 = __fadd2_rn(aL, nabs(t.a5)), t6 = __fadd2_rn(aL, nabs(t.a6));
    auto m = [](float a, float b, float c2, float d) {
        return fminf(fminf(fabsf(a), fabsf(b)), fminf(fabsf(c2), fabsf(d)));
    };
    return make_float2(m(t1.x, t2.x, t5.x, t6.x), m(t1.y, t2.y, t5.y, t6.y));
}

// select12 from the four differences t_j = |L| - |a_j| (computed by the caller) and Ls.
__device__ __forceinline__ float select12_t(float t1, float t2, float t5, float t6, float Ls) {
    float t = t1;
    t = fabsf(t2) < fabsf(t) ? t2 : t;
    t = fabsf(t5) < fabsf(t) ? t5 : t;
    t = fabsf(t6) < fabsf(t) ? t6 : t;
    return __int_as_float(__float_as_int(t) ^ (__float_as_int(Ls) & 0x80000000));
}
// The selection of two cells: the four differences |L| - |a_j| of both as packed FP32x2 adds (the
// same roundings as select12's scalar ones), the compare-select chain per lane.  The sign guard
// stays a scalar FMA per lane: one packed FMA for both lanes makes each selection wait for the
// other lane's operands and measured 1.3 % slower.
__device__ __forceinline__ float2 select12_x2(const Terms2 &t) {
    const float2 aL = make_float2(fabsf(t.L.x), fabsf(t.L.y));
    auto nabs = [](float2 v) { return make_float2(-fabsf(v.x), -fabsf(v.y)); };
    const float2 t1 = __fadd2_rn(aL, nabs(t.a1)), t2 = __fadd2_rn(aL, nabs(t.a2));
    const float2 t5 = __fadd2_rn(aL, nabs(t.a5)), t6 = __fadd2_rn(aL, nabs(t.a6));
    return make_float2(select12_t(t1.x, t2.x, t5.x, t6.x, fmaf(0x1p-40f, t.a1.x, t.L.x)),
                       select12_t(t1.y, t2.y, t5.y, t6.y, fmaf(0x1p-40f, t.a1.y, t.L.y)));
}

__device__ __forceinline__ float2 half_laplace12_x2(float2 nw, float2 n, float2 ne, float2 w,
                                                    float2 c, float2 e, float2 sw, float2 s,
                                                    float2 se) {
    return select12_x2(half_laplace12_terms_x2(nw, n, ne, w, c, e, sw, s, se));
}


// ---------------------------------------------------------------- storage types
template <typename S> struct Store;

// load/store: one element; load2/store2: two adjacent elements in one access (the address
// must be aligned to twice the element size).
template <> struct Store<float> {
    static __device__ __forceinline__ float load(const float *p) { return __ldg(p); }
    static __device__ __forceinline__ float to_float(float v) { return v; }
    static __device__ __forceinline__ float2 load2(const float *p) {
        return __ldg(reinterpret_cast<const float2 *>(p));
    }
    static __device__ __forceinline__ float round(float v) { return v; }
    static __device__ __forceinline__ float2 round2(float2 v) { return v; }
    static __device__ __forceinline__ void store(float *p, float v) { *p = v; }
    static __device__ __forceinline__ void store2(float *p, float a, float b) {
        *reinterpret_cast<float2 *>(p) = make_float2(a, b);
    }
};

template <> struct Store<__nv_bfloat16> {
    static __device__ __forceinline__ float load(const __nv_bfloat16 *p) {
        return __bfloat162float(__ldg(p));
    }
    static __device__ __forceinline__ float to_float(__nv_bfloat16 v) { return __bfloat162float(v); }
    static __device__ __forceinline__ float2 load2(const __nv_bfloat16 *p) {
        return __bfloat1622float2(__ldg(reinterpret_cast<const __nv_bfloat162 *>(p)));
    }
    static __device__ __forceinline__ float round(float v) {
        return __bfloat162float(__float2bfloat16_rn(v));
    }
    // both lanes rounded by one paired conversion (each to nearest even, as round())
    // two elements packed in 32 bits (lower address in the low half) widened to FP32
    static __device__ __forceinline__ float2 unpack2(uint32_t bits) {
        return make_float2(__uint_as_float(bits << 16), __uint_as_float(bits & 0xffff0000u));
    }
    static __device__ __forceinline__ float2 round2(float2 v) {
        const __nv_bfloat162 r = __floats2bfloat162_rn(v.x, v.y);
        uint32_t bits;
        memcpy(&bits, &r, sizeof bits);
        return unpack2(bits);  // widening a bfloat16 is a shift
    }
    static __device__ __forceinline__ void store(__nv_bfloat16 *p, float v) {
        *p = __float2bfloat16_rn(v);
    }
    static __device__ __forceinline__ void store2(__nv_bfloat16 *p, float a, float b) {
        *reinterpret_cast<__nv_bfloat162 *>(p) = __floats2bfloat162_rn(a, b);
    }
};

template <> struct Store<__half> {
    static __device__ __forceinline__ float load(const __half *p) { return __half2float(__ldg(p)); }
    static __device__ __forceinline__ float to_float(__half v) { return __half2float(v); }
    static __device__ __forceinline__ float2 load2(const __half *p) {
        return __half22float2(__ldg(reinterpret_cast<const __half2 *>(p)));
    }
    static __device__ __forceinline__ float round(float v) {
        return __half2float(__float2half_rn(v));
    }
    static __device__ __forceinline__ float2 round2(float2 v) {
        return __half22float2(__floats2half2_rn(v.x, v.y));
    }
    static __device__ __forceinline__ float2 unpack2(uint32_t bits) {
        __half2 hv;
        memcpy(&hv, &bits, sizeof bits);
        return __half22float2(hv);
    }
    static __device__ __forceinline__ void store(__half *p, float v) { *p = __float2half_rn(v); }
    static __device__ __forceinline__ void store2(__half *p, float a, float b) {
        *reinterpret_cast<__half2 *>(p) = __floats2half2_rn(a, b);
    }
};

enum Boundary { BND_REPLICATE = 0, BND_ZERO = 1 };

}  // namespace wmc
