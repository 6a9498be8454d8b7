// kd_dw.cuh -- double-word FP32 arithmetic for the FP64-accurate form of the
// split-operator step (KD_DW).  A real number is the unevaluated sum h + l of two floats
// with |l| <= ulp(h)/2, which carries 48 significand bits (relative rounding unit
// 2^-48 = 3.6e-15): on GB300 the FP32 pipe issues 64x the FP64 pipe's operations, so a
// few FP32 operations per double-word operation are far cheaper than native FP64.
//
// Building blocks (published error-free transformations, written from their definitions):
//  - TwoSum (Knuth): s + e = a + b exactly, s = fl(a + b), 6 operations, any a, b;
//  - Fast2Sum (Dekker): the same in 3 operations when |a| >= |b| (or a = 0);
//  - TwoProd with FMA: p + e = a b exactly, p = fl(a b), 2 operations;
//  - the double-word sum of two double-words (Joldes, Muller & Popescu, 2017): the
//    "sloppy" form, relative error unbounded only under cancellation but absolute error
//    at most ~2^-47 (|x| + |y|), which is the bound an FFT's error analysis uses, 11 ops;
//  - double-word times double-word with FMA, relative error ~5 2^-48, 7 ops;
//  - double-word times float, 5 ops.
// No operation here is contracted or reassociated by the compiler: every one is written
// with the rounding it needs (__fadd_rn, __fmul_rn, __fmaf_rn), so the error-free
// transformations stay exact under -O3.
#pragma once
#include <cuda_runtime.h>

namespace kd {

struct DW {
    float h, l;
};

#define KD_DWI __host__ __device__ __forceinline__

#ifdef __CUDA_ARCH__
KD_DWI float f_add(float a, float b) { return __fadd_rn(a, b); }
KD_DWI float f_sub(float a, float b) { return __fsub_rn(a, b); }
KD_DWI float f_mul(float a, float b) { return __fmul_rn(a, b); }
KD_DWI float f_fma(float a, float b, float c) { return __fmaf_rn(a, b, c); }
#else
KD_DWI float f_add(float a, float b) { volatile float s = a + b; return s; }
KD_DWI float f_sub(float a, float b) { volatile float s = a - b; return s; }
KD_DWI float f_mul(float a, float b) { volatile float s = a * b; return s; }
KD_DWI float f_fma(float a, float b, float c) { return fmaf(a, b, c); }
#endif

KD_DWI DW two_sum(float a, float b) {
    const float s = f_add(a, b);
    const float bb = f_sub(s, a);
    const float e = f_add(f_sub(a, f_sub(s, bb)), f_sub(b, bb));
    return DW{s, e};
}
KD_DWI DW fast_two_sum(float a, float b) {   // |a| >= |b| or a == 0
    const float s = f_add(a, b);
    return DW{s, f_sub(b, f_sub(s, a))};
}
KD_DWI DW two_prod(float a, float b) {
    const float p = f_mul(a, b);
    return DW{p, f_fma(a, b, -p)};
}

KD_DWI DW dw(float a) { return DW{a, 0.0f}; }
// 2^-m for 0 <= m <= 126, exact
KD_DWI float pow2_neg(int m) {
#ifdef __CUDA_ARCH__
    return __int_as_float((127 - m) << 23);
#else
    return ldexpf(1.0f, -m);
#endif
}
KD_DWI DW dw_neg(DW x) { return DW{-x.h, -x.l}; }
// x * 2^k for a power-of-two float p (exact)
KD_DWI DW dw_scale(DW x, float p) { return DW{x.h * p, x.l * p}; }

// x + y (sloppy double-word sum): absolute error <= ~2^-47 (|x| + |y|)
KD_DWI DW dw_add(DW x, DW y) {
    const DW s = two_sum(x.h, y.h);
    const float v = f_add(x.l, y.l);
    const float w = f_add(s.l, v);
    return fast_two_sum(s.h, w);
}
KD_DWI DW dw_sub(DW x, DW y) { return dw_add(x, dw_neg(y)); }
// Lazy sums for a butterfly's first level: x + y as (h, l) with h = fl(x.h + y.h) exact to
// its TwoSum error and l = that error plus both low parts, not renormalised (|l| may exceed
// half an ulp of h).  dw_add_lazy then adds two such pairs and renormalises once: the
// result has the sloppy double-word sum's absolute error bound (a few 2^-48 of the summed
// magnitudes) with one Fast2Sum instead of three.
KD_DWI DW dw_add_part(DW x, DW y) {
    const DW s = two_sum(x.h, y.h);
    return DW{s.h, f_add(s.l, f_add(x.l, y.l))};
}
KD_DWI DW dw_add_lazy(DW x, DW y) {
    const DW s = two_sum(x.h, y.h);
    return fast_two_sum(s.h, f_add(s.l, f_add(x.l, y.l)));
}
// x + y with y a float
KD_DWI DW dw_add_f(DW x, float y) {
    const DW s = two_sum(x.h, y);
    return fast_two_sum(s.h, f_add(s.l, x.l));
}
// x * y, both double-words (FMA form): relative error <= ~5 2^-48
KD_DWI DW dw_mul(DW x, DW y) {
    const DW c = two_prod(x.h, y.h);
    const float t = f_fma(x.l, y.h, f_mul(x.h, y.l));
    return fast_two_sum(c.h, f_add(c.l, t));
}
// x * y with y a float: relative error <= ~2 2^-48
KD_DWI DW dw_mul_f(DW x, float y) {
    const DW c = two_prod(x.h, y);
    return fast_two_sum(c.h, f_fma(x.l, y, c.l));
}
// a x + b y as one double-word (the real part of a complex product): the two leading
// products exactly, their sum by TwoSum, every small term gathered in one float
KD_DWI DW dw_dot2(DW a, DW x, DW b, DW y) {
    const DW p = two_prod(a.h, x.h);
    const DW q = two_prod(b.h, y.h);
    const DW s = two_sum(p.h, q.h);
    float t = f_add(p.l, q.l);
    t = f_add(t, s.l);
    t = f_fma(a.h, x.l, t);
    t = f_fma(a.l, x.h, t);
    t = f_fma(b.h, y.l, t);
    t = f_fma(b.l, y.h, t);
    return fast_two_sum(s.h, t);
}

// The same dot product without the final renormalisation (|l| may exceed half an ulp of
// h): for values that go straight into a butterfly's first level (dw_add_part / dw_add),
// whose TwoSum of the high parts is exact whatever the low parts are
KD_DWI DW dw_dot2_part(DW a, DW x, DW b, DW y) {
    const DW p = two_prod(a.h, x.h);
    const DW q = two_prod(b.h, y.h);
    const DW s = two_sum(p.h, q.h);
    float t = f_add(p.l, q.l);
    t = f_add(t, s.l);
    t = f_fma(a.h, x.l, t);
    t = f_fma(a.l, x.h, t);
    t = f_fma(b.h, y.l, t);
    t = f_fma(b.l, y.h, t);
    return DW{s.h, t};
}

// Splits a double into the nearest double-word (exact for the 48 leading bits); host or
// device, FP64.
KD_DWI DW dw_from_double(double d) {
    const float h = (float)d;
    const float l = (float)(d - (double)h);
    return DW{h, l};
}
KD_DWI double dw_to_double(DW x) { return (double)x.h + (double)x.l; }

KD_DWI DW operator+(DW x, DW y) { return dw_add(x, y); }
KD_DWI DW operator-(DW x, DW y) { return dw_sub(x, y); }
KD_DWI DW operator-(DW x) { return dw_neg(x); }
KD_DWI DW operator*(DW x, DW y) { return dw_mul(x, y); }
// sign factor +-1 (the FFT direction) times x: exact
KD_DWI DW operator*(int sgn, DW x) { return sgn > 0 ? x : dw_neg(x); }

// sqrt(x) for x >= 0: float seed and one correction, relative error ~2^-47
KD_DWI DW dw_sqrt(DW x) {
    if (!(x.h > 0.0f)) return DW{0.0f, 0.0f};
    const float r = sqrtf(x.h);
    const DW r2 = two_prod(r, r);
    const float d = f_add(f_sub(f_sub(x.h, r2.h), r2.l), x.l);
    return fast_two_sum(r, d / (2.0f * r));
}
// x / y: float quotient and one correction from the double-word remainder
KD_DWI DW dw_div(DW x, DW y) {
    const float q = x.h / y.h;
    const DW r = dw_sub(x, dw_mul_f(y, q));
    return fast_two_sum(q, r.h / y.h);
}

// Constant tables of the double-word transcendental functions, built once per
// simulation in FP64 (kd_api.cu) and passed to the kernels:
//   sc[j + 13], j = -13..13: (sin(j/16).h, sin(j/16).l, cos(j/16).h, cos(j/16).l);
//   e2[j], j = 0..31: (2^(-j/32).h, 2^(-j/32).l).
struct DWConst {
    float4 sc[27];
    float2 e2[32];
};

// exp(-u) for u >= 0 (e^-u below 1e-34 returns 0).  Range reduction u = n ln2/32 + r with
// |r| <= ln2/64 (Cody-Waite: ln2/32 = L1 + L2, L1 with 12 significant bits so that n L1
// is exact), e^-u = 2^(-n div 32) 2^(-(n mod 32)/32) e^-r; e^-r = 1 + x + x^2 (1/2 + t(x)),
// x = -r, with the tail t = x/6 + x^2/24 + x^3/120 + x^4/720 in FP32 (below 3e-7 in size,
// so its rounding stays under 1e-14 of the result).  Relative error ~1e-14.
KD_DWI DW dw_exp_neg(DW u, const DWConst* K) {
    if (!(u.h < 78.0f)) return DW{0.0f, 0.0f};
    const float L1 = 0.02166748046875f;                       // 355 / 2^14
    const DW L2 = DW{-6.6310763e-06f, 5.1455368e-14f};        // ln2/32 - L1
    const float n = rintf(u.h * 46.166241308446828f);          // u 32/ln2
    DW r = dw_add_f(u, -n * L1);
    r = dw_sub(r, dw_mul_f(L2, n));
    const DW x = dw_neg(r);
    const float xf = x.h;
    const float t = xf * (1.0f / 6 + xf * (1.0f / 24 + xf * (1.0f / 120 + xf * (1.0f / 720))));
    const DW x2 = dw_mul(x, x);
    DW e = dw_add(dw_add_f(x, 1.0f), dw_mul(x2, dw_add_f(DW{0.5f, 0.0f}, t)));
    const int ni = (int)n;
    const int j = ni & 31, m = ni >> 5;
    const float2 c = K->e2[j];
    e = dw_mul(e, DW{c.x, c.y});
    return dw_scale(e, pow2_neg(m));
}

// sin and cos of a double-word angle |th| <= 2^10: quadrant reduction th = r + q pi/2
// (Cody-Waite with pi/2 = P1 + P2, P1 with 12 significant bits), table step
// r = j/16 + r', |r'| <= 1/32, Taylor series of r' (the leading terms in double-word, the
// tails in FP32), and the angle-addition formulas.  Relative error ~1e-14.
KD_DWI void dw_sincos(DW th, const DWConst* K, DW* sn, DW* cs) {
    const float P1 = 1.57080078125f;                           // 3217 / 2^11
    const DW P2 = DW{-4.454455e-06f, -1.6520119e-13f};        // pi/2 - P1
    const float q = rintf(th.h * 0.63661977236758134f);
    DW r = dw_add_f(th, -q * P1);
    r = dw_sub(r, dw_mul_f(P2, q));
    const float jf = rintf(r.h * 16.0f);
    const DW rp = dw_add_f(r, -jf * 0.0625f);
    const DW s2 = dw_mul(rp, rp);
    const float sf = s2.h;
    // sin r' = r' (1 + s2 (-1/6 + s2 (1/120 - s2/5040 + s2^2/362880)))
    const float ts = sf * (1.0f / 120 + sf * (-1.0f / 5040 + sf * (1.0f / 362880)));
    const DW sr = dw_mul(rp, dw_add_f(dw_mul(s2, dw_add_f(DW{-1.6666667e-01f, 4.967054e-09f}, ts)), 1.0f));
    // cos r' = 1 + s2 (-1/2 + s2 (1/24 - s2/720 + s2^2/40320))
    const float tc = sf * (0.041666667908430099f + sf * (-1.0f / 720 + sf * (1.0f / 40320)));
    const DW cr = dw_add_f(dw_mul(s2, dw_add_f(DW{-0.5f, 0.0f}, tc)), 1.0f);
    const float4 t = K->sc[(int)jf + 13];
    const DW S = DW{t.x, t.y}, C = DW{t.z, t.w};
    const DW s0 = dw_dot2(S, cr, C, sr);            // sin(j/16 + r')
    const DW c0 = dw_dot2(C, cr, dw_neg(S), sr);    // cos(j/16 + r')
    const int qi = ((int)q) & 3;
    *sn = qi == 0 ? s0 : qi == 1 ? c0 : qi == 2 ? dw_neg(s0) : dw_neg(c0);
    *cs = qi == 0 ? c0 : qi == 1 ? dw_neg(s0) : qi == 2 ? dw_neg(c0) : s0;
}

// ------------------------------------------------------------ complex double-word -
// members named x, y like float2/double2, so the FFT engine's generic complex code applies
struct DWC {
    DW x, y;
};
KD_DWI DWC dwc(DW re, DW im) { return DWC{re, im}; }
KD_DWI DWC dwc_add(DWC a, DWC b) { return DWC{dw_add(a.x, b.x), dw_add(a.y, b.y)}; }
KD_DWI DWC dwc_sub(DWC a, DWC b) { return DWC{dw_sub(a.x, b.x), dw_sub(a.y, b.y)}; }
// a * w, w = (c, s): (a.x c - a.y s, a.x s + a.y c)
KD_DWI DWC dwc_mul(DWC a, DWC w) {
    return DWC{dw_dot2(a.x, w.x, dw_neg(a.y), w.y), dw_dot2(a.x, w.y, a.y, w.x)};
}
// a * w unnormalised (dw_dot2_part): the FFT's twiddle products, which feed the next
// butterfly directly
KD_DWI DWC dwc_mul_part(DWC a, DWC w) {
    return DWC{dw_dot2_part(a.x, w.x, dw_neg(a.y), w.y), dw_dot2_part(a.x, w.y, a.y, w.x)};
}
// a * r for a real double-word r
KD_DWI DWC dwc_mul_r(DWC a, DW r) { return DWC{dw_mul(a.x, r), dw_mul(a.y, r)}; }

}  // namespace kd
