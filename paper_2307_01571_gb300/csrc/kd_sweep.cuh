// kd_sweep.cuh -- the fused sweep kernels of the FFT split-operator step (Sec. II.D of
// arXiv 2307.01571) for sm_103a.
//
// One Strang step psi <- V_half(t_{n+1}) F^-1 K F V_half(t_n) psi is executed as two
// passes over the spinor in HBM:
//   x sweep: per row  -- inverse x-FFT, merged potential factor exp(-i dt V(t_n)/hbar)
//            (closing half of step n-1 times opening half of step n, the same matrix),
//            forward x-FFT;
//   y sweep: per column tile -- forward y-FFT, kinetic factor, inverse y-FFT.
// Between sweeps the state lives in (k_x, y) space.  The first and last x sweeps of a
// run apply a true half step and only one of the two FFTs.
//
// FFT engine: Stockham autosort, radix 8/4/2, every thread owns E = 8 (FP32) or 4 (FP64)
// elements of one line for all four spinor components in registers; butterflies run on
// registers and stages exchange data through shared memory with an XOR swizzle that
// keeps 16-byte accesses free of bank conflicts.  The last stage of the first FFT and the
// first stage of the second FFT use the same radix and butterfly-to-thread map, so the
// pointwise factor in between is applied straight on registers with no exchange, and the
// first/last stages read/write global memory in natural order (coalesced, in place).
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include <type_traits>

#include "kd_dw.cuh"
#include "kd_internal.h"

namespace kd {

#define KD_DI __device__ __forceinline__

template <typename T> struct Cx;
template <> struct Cx<float> { using t = float2; };
template <> struct Cx<double> { using t = double2; };
template <> struct Cx<DW> { using t = DWC; };

template <typename C> KD_DI C mk(decltype(C::x) a, decltype(C::x) b) { C r; r.x = a; r.y = b; return r; }
template <typename C> KD_DI C cadd(C a, C b) { return mk<C>(a.x + b.x, a.y + b.y); }
template <typename C> KD_DI C csub(C a, C b) { return mk<C>(a.x - b.x, a.y - b.y); }
template <typename C> KD_DI C cmul(C a, C b) {
    return mk<C>(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
// a times (DIR i)
template <int DIR, typename C> KD_DI C mul_i(C a) {
    return DIR > 0 ? mk<C>(-a.y, a.x) : mk<C>(a.y, -a.x);
}

// ------------------------------------------------------------ small DFTs ---------
// In place on a[0], a[S], ..., output in natural order, X_k = sum_j a_j w^{jk},
// w = exp(DIR 2 pi i / R).
template <int DIR, int S, typename C> KD_DI void dft2(C* a) {
    C t = a[0];
    a[0] = cadd(t, a[S]);
    a[S] = csub(t, a[S]);
}

template <int DIR, int S, typename C> KD_DI void dft4(C* a) {
    C s02 = cadd(a[0], a[2 * S]), d02 = csub(a[0], a[2 * S]);
    C s13 = cadd(a[S], a[3 * S]), d13 = csub(a[S], a[3 * S]);
    C r = mul_i<DIR>(d13);
    a[0] = cadd(s02, s13);
    a[2 * S] = csub(s02, s13);
    a[S] = cadd(d02, r);
    a[3 * S] = csub(d02, r);
}

// The same four-point DFT on double-word values: the first level's sums and differences
// stay unnormalised (dw_add_part) and each output renormalises once (dw_add_lazy)
template <int DIR, int S> KD_DI void dft4(DWC* a) {
    const DW s02x = dw_add_part(a[0].x, a[2 * S].x), s02y = dw_add_part(a[0].y, a[2 * S].y);
    const DW d02x = dw_add_part(a[0].x, dw_neg(a[2 * S].x)), d02y = dw_add_part(a[0].y, dw_neg(a[2 * S].y));
    const DW s13x = dw_add_part(a[S].x, a[3 * S].x), s13y = dw_add_part(a[S].y, a[3 * S].y);
    const DW d13x = dw_add_part(a[S].x, dw_neg(a[3 * S].x)), d13y = dw_add_part(a[S].y, dw_neg(a[3 * S].y));
    // r = (DIR i) d13
    const DW rx = DIR > 0 ? dw_neg(d13y) : d13y, ry = DIR > 0 ? d13x : dw_neg(d13x);
    a[0] = DWC{dw_add_lazy(s02x, s13x), dw_add_lazy(s02y, s13y)};
    a[2 * S] = DWC{dw_add_lazy(s02x, dw_neg(s13x)), dw_add_lazy(s02y, dw_neg(s13y))};
    a[S] = DWC{dw_add_lazy(d02x, rx), dw_add_lazy(d02y, ry)};
    a[3 * S] = DWC{dw_add_lazy(d02x, dw_neg(rx)), dw_add_lazy(d02y, dw_neg(ry))};
}

// multiply by 1/sqrt(2) as a hi + lo pair: a single rounded constant would make every
// radix-8 butterfly shrink the norm of two of its eight inputs by 2 h^2 - 1 (about 4e-8
// in FP32), a bias that accumulates over thousands of steps
template <typename T> KD_DI T mul_rsqrt2(T x) {
    if constexpr (std::is_same<T, DW>::value) {
        return dw_mul(x, DW{0.707106769f, 1.21016175e-08f});
    } else if constexpr (sizeof(T) == 4) {
        return fmaf(x, 0.707106769084930419921875f, x * 1.2101617e-08f);
    } else {
        return fma(x, 0.70710678118654757, x * -4.8336466567264567e-17);
    }
}

template <int DIR, int S, typename C> KD_DI void dft8(C* a) {
    C e[4] = {a[0], a[2 * S], a[4 * S], a[6 * S]};
    C o[4] = {a[S], a[3 * S], a[5 * S], a[7 * S]};
    dft4<DIR, 1>(e);
    dft4<DIR, 1>(o);
    // o_k *= w8^k, w8 = exp(DIR 2 pi i / 8)
    o[1] = mk<C>(mul_rsqrt2(o[1].x - DIR * o[1].y), mul_rsqrt2(o[1].y + DIR * o[1].x));
    o[2] = mul_i<DIR>(o[2]);
    o[3] = mk<C>(mul_rsqrt2(-o[3].x - DIR * o[3].y), mul_rsqrt2(-o[3].y + DIR * o[3].x));
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        a[k * S] = cadd(e[k], o[k]);
        a[(k + 4) * S] = csub(e[k], o[k]);
    }
}

template <int R, int DIR, int S, typename C> KD_DI void dftR(C* a) {
    if constexpr (R == 2) dft2<DIR, S>(a);
    else if constexpr (R == 4) dft4<DIR, S>(a);
    else dft8<DIR, S>(a);
}

// ------------------------------------------------------------- plan ---------------
// Radix plan of an N = 2^logn point FFT with maximum radix 2^loge: as many radix-2^loge
// stages as fit, the remainder as radix-4 or radix-2 stages.
__host__ __device__ constexpr int plan_nst(int logn, int loge) {
    return loge == 3 ? (logn % 3 == 0 ? logn / 3 : logn / 3 + 1)
                     : (loge == 2 ? logn / 2 + logn % 2 : logn);
}
__host__ __device__ constexpr int plan_logr(int logn, int loge, int s) {
    if (loge == 3) {
        int q = logn / 3, r = logn % 3;
        if (r == 0) return 3;
        if (r == 1) return s < q - 1 ? 3 : 2;
        return s < q ? 3 : 2;
    }
    if (loge == 2) return s < logn / 2 ? 2 : 1;
    return 1;
}
__host__ __device__ constexpr int plan_logns(int logn, int loge, int s) {  // log2 of Ns before stage s
    int a = 0;
    for (int i = 0; i < s; ++i) a += plan_logr(logn, loge, i);
    return a;
}
// Twiddle table layout: stage-major, one segment per stage order (plan order, then
// reversed order), stages in execution order, entries [r - 1][k] for r = 1..R-1 and
// k = 0..Ns-1, value exp(-2 pi i r k / (Ns R)).  A warp's lanes have consecutive k, so
// every twiddle load is contiguous (or a broadcast when Ns < 32).
__host__ __device__ constexpr int stage_lns(int logn, int loge, bool rev, int S) {
    return rev ? logn - plan_logns(logn, loge, plan_nst(logn, loge) - S) : plan_logns(logn, loge, S);
}
__host__ __device__ constexpr int stage_lr(int logn, int loge, bool rev, int S) {
    return plan_logr(logn, loge, rev ? plan_nst(logn, loge) - 1 - S : S);
}
__host__ __device__ constexpr int stage_tw_entries(int logn, int loge, bool rev, int S) {
    return stage_lns(logn, loge, rev, S) > 0
               ? ((1 << stage_lr(logn, loge, rev, S)) - 1) << stage_lns(logn, loge, rev, S)
               : 0;
}
__host__ __device__ constexpr int tw_offset(int logn, int loge, bool rev, int S) {
    int off = 0;
    if (rev)
        for (int i = 0; i < plan_nst(logn, loge); ++i) off += stage_tw_entries(logn, loge, false, i);
    for (int i = 0; i < S; ++i) off += stage_tw_entries(logn, loge, rev, i);
    return off;
}
__host__ __device__ constexpr int tw_total(int logn, int loge) {
    return tw_offset(logn, loge, true, plan_nst(logn, loge));
}

__host__ __device__ constexpr int cmin(int a, int b) { return a < b ? a : b; }
__host__ __device__ constexpr int cmax(int a, int b) { return a > b ? a : b; }
__host__ __device__ constexpr int clog2(int v) { return v <= 1 ? 0 : 1 + clog2(v / 2); }

template <typename T, int LOGN, int AXIS, int V> struct Cfg {
    static constexpr bool F64 = sizeof(T) == 8;                  // FP64 or double-word
    static constexpr bool DWT = std::is_same<T, DW>::value;      // double-word form
    static constexpr SweepVariant VS = sweep_variant(AXIS, F64 ? 0 : V);
    static constexpr int N = 1 << LOGN;
    // components per thread: the double-word form keeps one pair per thread (its
    // arithmetic needs many registers) and shares the field between the pairs of a CTA
    static constexpr int NC = DWT ? 2 : sweep_nc(F64, AXIS, LOGN, V);
    static constexpr int LOGE = DWT ? sweep_loge_dw(LOGN) : sweep_loge(F64, AXIS, LOGN, V);
    static constexpr int E = 1 << LOGE;                          // elements per thread
    static constexpr int TF = N / E;                             // threads per line
    // lines per CTA: rows are batched up to the variant's thread count; column tiles take
    // that many threads and at least MINB columns (FP64: 2), i.e. >= 64-128 contiguous
    // bytes per tile row, within 512 threads
    static constexpr int MINB = F64 ? 2 : VS.minb;
    // field sharing between the two pairs of a line (x axis, one pair per thread)
    static constexpr bool SHARE = AXIS == AXIS_X && NC == 2 && TF <= 256 &&
                                  (DWT || (!F64 && VS.share != 0));
    static constexpr int PCTA = SHARE ? 2 : 1;                  // pairs per CTA (NC = 2)
    static constexpr int BATCH = AXIS == AXIS_X ? cmax(1, (DWT ? 256 : F64 ? 128 : VS.threads) / PCTA / TF)
                                                : (TF * MINB > 512 ? cmax(1, 512 / TF)
                                                                   : cmax(MINB, (F64 ? 256 : VS.threads) / TF));
    static constexpr int THREADS = TF * BATCH * PCTA;
    static constexpr int CPP = F64 ? 1 : 2;                      // complex per 16-byte unit
    static constexpr int NPL = NC / CPP;                         // units per point in the CTA
    static constexpr int PPP = 2 / CPP;                          // units per point per pair
    static constexpr int NPAIRS = SHARE ? 1 : 4 / NC;            // CTAs per line group
    static constexpr int NST = plan_nst(LOGN, LOGE);
    static constexpr int BUF_UNITS = PCTA * BATCH * NPL * N;     // one exchange buffer
    // resident CTAs per SM the FP32 sweeps are built for (the variant's resident warps;
    // the default puts the 1024x512 grid's lines in one wave); FP64 sweeps keep their full
    // register budget
    static constexpr int MINBLK = DWT ? cmax(1, 16 * 32 / THREADS)
                                      : (F64 ? 1 : cmax(1, VS.resident_warps * 32 / THREADS));
    // two exchange buffers (one barrier per exchange) only when they keep that occupancy
    static constexpr bool DB = 2 * BUF_UNITS * 16 * MINBLK <= 200 * 1024;
    static constexpr int SMEM_BYTES = cmax(NST > 1 ? (DB ? 2 : 1) * BUF_UNITS * 16 : 16,
                                           SHARE ? BATCH * N * (DWT ? 32 : 16) : 16);
    // lanes of one 8-lane (128-byte) shared-memory wavefront cover 2^LOGG consecutive
    // butterflies
    static constexpr int LOGG =
        cmin(LOGN, AXIS == AXIS_X ? 3 : cmax(0, 3 - clog2(BATCH)));
};

// XOR swizzle of element index i for the exchange after a stage with Ns = 2^la and
// radix 2^lb: spreads the 2^g butterflies of a wavefront over distinct 16-byte bank
// groups for the strided write and keeps the contiguous read conflict-free.  The map is
// linear over GF(2) (swz(a ^ b) = swz(a) ^ swz(b)), which the exchange uses to reduce
// every access to one XOR of a per-thread base with a compile-time constant.
template <int LA, int LB, int G> __host__ __device__ constexpr int swz(int i) {
    if constexpr (LA >= G) {
        return i;
    } else {
        constexpr int SH = cmax(G, LA + LB);
        constexpr int W = cmin(LB, G - LA);
        return i ^ (((i >> SH) & ((1 << W) - 1)) << LA);
    }
}
// Stockham output index of butterfly j before adding r Ns: (j / Ns) Ns R + j mod Ns
// (also GF(2)-linear in j)
template <int LA, int LB> __host__ __device__ constexpr int expand(int j) {
    return ((j >> LA) << (LA + LB)) | (j & ((1 << LA) - 1));
}

// ------------------------------------------------------- register <-> 16 B --------
template <typename T> struct Unit;
template <> struct Unit<float> {
    using U = float4;
    KD_DI static U pack(const float2* c) { return make_float4(c[0].x, c[0].y, c[1].x, c[1].y); }
    KD_DI static void unpack(U u, float2* c) { c[0] = make_float2(u.x, u.y); c[1] = make_float2(u.z, u.w); }
};
template <> struct Unit<double> {
    using U = double2;
    KD_DI static U pack(const double2* c) { return c[0]; }
    KD_DI static void unpack(U u, double2* c) { c[0] = u; }
};
// double-word complex: (re.h, re.l, im.h, im.l), each real in the 8 bytes a double would take
template <> struct Unit<DW> {
    using U = float4;
    KD_DI static U pack(const DWC* c) { return make_float4(c[0].x.h, c[0].x.l, c[0].y.h, c[0].y.l); }
    KD_DI static void unpack(U u, DWC* c) { c[0] = DWC{DW{u.x, u.y}, DW{u.z, u.w}}; }
};

// ------------------------------------------------- double-word potential factor ---
// The potential factor exp(-i tau V/hbar) at one point in double-word arithmetic,
// returned as (cos theta - 1, s a_y, s a_x) with s = sin(theta)/|a|, theta = kappa |a|:
// the standing wave of Eqs. (Equation_of_Gaussian_beam) in product form (see
// Sweep::op_potential_std), every quantity a double-word and exp, sin, cos of kd_dw.cuh
// (relative error ~1e-14 of the field).  Table xtab holds per column x two double-word
// 4-vectors (Theta0, x/(x_R w^2), w0/w, 1/w^2) and (1/w, cos zeta, sin zeta, cos k x) as
// float4 [2][nx][2].  Not inlined: the kernels call it once per point, and one copy per
// kernel keeps compile time and code size down.
struct DWFactor {
    DW c1, say, sax;
};
static __device__ __noinline__ DWFactor dw_potential_factor(const void* xtab_, const void* dwconst, int nx, int x,
                                                     int kind, int longitudinal, DW y, DW y2, DW st,
                                                     DW kap, DW e4) {
    const DWConst* K = reinterpret_cast<const DWConst*>(dwconst);
    const float4* xt = reinterpret_cast<const float4*>(xtab_);
    const float4 q2 = __ldg(xt + 2 * (nx + x));       // 1/w, cos zeta
    const float4 q3 = __ldg(xt + 2 * (nx + x) + 1);   // sin zeta, cos k x
    DW ax = DW{0.0f, 0.0f}, ay;
    if (kind == 1) {
        ay = dw_scale(dw_mul(st, DW{q3.z, q3.w}), -2.0f);
    } else {
        const float4 q0 = __ldg(xt + 2 * x);          // Theta0, x/(x_R w^2)
        const float4 q1 = __ldg(xt + 2 * x + 1);      // w0/w, 1/w^2
        const DW G = dw_mul(DW{q1.x, q1.y}, dw_exp_neg(dw_mul(DW{q1.z, q1.w}, y2), K));
        const DW th = dw_sub(DW{q0.x, q0.y}, dw_mul(DW{q0.z, q0.w}, y2));
        DW sn, cs;
        dw_sincos(th, K, &sn, &cs);
        const DW sg = dw_mul(st, G);
        ay = dw_scale(dw_mul(sg, cs), -2.0f);
        if (longitudinal)
            ax = dw_mul(dw_mul(e4, sg), dw_mul(dw_mul(y, DW{q2.x, q2.y}),
                                               dw_dot2(sn, DW{q2.z, q2.w}, cs, DW{q3.x, q3.y})));
    }
    const DW a2 = dw_dot2(ax, ax, ay, ay);
    const DW th2 = dw_mul(dw_mul(kap, kap), a2);
    DW c1, s;
    if (th2.h < 0.0625f) {
        // Taylor series in theta^2: the terms above 1e-8 in double-word, the tails in FP32
        const float t2 = th2.h;
        const float tc = t2 * (-1.0f / 720 + t2 * (1.0f / 40320 + t2 * (-1.0f / 3628800)));
        c1 = dw_mul(th2, dw_add_f(dw_mul(th2, dw_add_f(DW{4.16666679e-02f, -1.24176339e-09f}, tc)), -0.5f));
        const float ts = t2 * (-1.0f / 5040 + t2 * (1.0f / 362880 + t2 * (-1.0f / 39916800)));
        const DW inner = dw_add(dw_mul(th2, dw_add_f(DW{8.33333377e-03f, -4.34617218e-10f}, ts)),
                                DW{-1.66666672e-01f, 4.96705388e-09f});
        s = dw_mul(kap, dw_add_f(dw_mul(th2, inner), 1.0f));
    } else {
        const DW amag = dw_sqrt(a2);
        DW sh, ch;
        dw_sincos(dw_scale(dw_mul(kap, amag), 0.5f), K, &sh, &ch);
        c1 = dw_scale(dw_mul(sh, sh), -2.0f);
        s = dw_div(dw_scale(dw_mul(sh, ch), 2.0f), amag);
    }
    return DWFactor{c1, dw_mul(s, ay), dw_mul(s, ax)};
}

// ------------------------------------------------------------- the kernel ---------
template <typename T, int LOGN, int AXIS, int SHAPE, int V> struct Sweep {
    using Cf = Cfg<T, LOGN, AXIS, V>;
    using C = typename Cx<T>::t;
    using U = typename Unit<T>::U;
    static constexpr int N = Cf::N, E = Cf::E, TF = Cf::TF, NC = Cf::NC, NST = Cf::NST;
    static constexpr bool DWF = std::is_same<T, DW>::value;   // double-word form
    static constexpr int NPL = Cf::NPL, CPP = Cf::CPP, BATCH = Cf::BATCH;
    // direction of the first and second FFT (forward = -1)
    static constexpr int DIR1 = AXIS == AXIS_X ? +1 : -1;
    static constexpr int DIR2 = -DIR1;
    static constexpr bool HAS1 = (SHAPE & SHAPE_F1) != 0;
    static constexpr bool HAS2 = (SHAPE & SHAPE_F2) != 0;
    // radix (log) of the stage that sits next to the pointwise op in both FFTs
    static constexpr int LR_OP = plan_logr(LOGN, Cf::LOGE, NST - 1);
    static constexpr int LR_LOAD = HAS1 ? plan_logr(LOGN, Cf::LOGE, 0) : LR_OP;
    static constexpr int LR_STORE = HAS2 ? plan_logr(LOGN, Cf::LOGE, 0) : LR_OP;

    struct Ctx {
        int jt, bb, line, pair;
        int n_local;   // step of the current kd_step call the potential factor is taken at
        int bar;       // barrier of the block's threads: 0 = the CTA's (see block_sync)
        bool valid;
        U* sm;
    };

    // barrier of the THREADS threads that run one launch block: the CTA's own barrier in
    // a standalone launch (bar 0, known at compile time there); a named barrier per block
    // where several blocks share a CTA (the persistent batch kernel), so that they do not
    // wait for each other
    KD_DI static void block_sync(const Ctx& c) {
        if (c.bar == 0) __syncthreads();
        else asm volatile("bar.sync %0, %1;" ::"r"(c.bar), "n"(Cf::THREADS) : "memory");
    }

    KD_DI static int point_of(const SweepArgs& a, int line, int idx) {
        return AXIS == AXIS_X ? line * a.nx + idx : idx * a.nx + line;
    }
    // spinor memory: two pair planes [pair][ny][nx][2 complex]; plane p of this CTA
    KD_DI static long long unit_of(const SweepArgs& a, const Ctx& c, long long pt, int p) {
        const int pair = NC == 4 ? p / Cf::PPP : c.pair;
        const int u = p % Cf::PPP;
        return ((long long)pair * a.nx * a.ny + pt) * Cf::PPP + u;
    }

    // registers hold slots e = m*R + r for butterfly j = jt + m*TF, element index
    // j + r*N/R (the input layout of a stage with radix R = 2^LR)
    template <int LR> KD_DI static void load(const SweepArgs& a, const Ctx& c, C* v) {
        constexpr int R = 1 << LR;
        const U* g = reinterpret_cast<const U*>(a.in);
#pragma unroll
        for (int m = 0; m < E / R; ++m)
#pragma unroll
            for (int r = 0; r < R; ++r) {
                int idx = c.jt + m * TF + r * (N / R);
                const long long pt = point_of(a, c.line, idx);
#pragma unroll
                for (int p = 0; p < NPL; ++p) {
                    U u;
                    // the spinor streams through L2 only (.cg), so that the small,
                    // reused twiddle and field tables stay resident in L1
                    if (c.valid) u = __ldcg(g + unit_of(a, c, pt, p));
                    else u = U{};
                    Unit<T>::unpack(u, v + (m * R + r) * NC + p * CPP);
                }
            }
    }
    template <int LR> KD_DI static void store(const SweepArgs& a, const Ctx& c, const C* v) {
        constexpr int R = 1 << LR;
        U* g = reinterpret_cast<U*>(a.out);
        if (!c.valid) return;
#pragma unroll
        for (int m = 0; m < E / R; ++m)
#pragma unroll
            for (int r = 0; r < R; ++r) {
                int idx = c.jt + m * TF + r * (N / R);
                const long long pt = point_of(a, c.line, idx);
#pragma unroll
                for (int p = 0; p < NPL; ++p) __stcg(g + unit_of(a, c, pt, p), Unit<T>::pack(v + (m * R + r) * NC + p * CPP));
            }
    }

    // one Stockham stage: twiddle (Ns > 1) and radix-R butterflies on registers
    // one Stockham stage: twiddle (Ns > 1) and radix-R butterflies on registers; the
    // stage's twiddles start at entry TWOFF of the stage-major table
    template <int DIR, int LR, int LNS, int TWOFF> KD_DI static void stage(const SweepArgs& a, const Ctx& c, C* v) {
        constexpr int R = 1 << LR;
        constexpr int NS = 1 << LNS;
#pragma unroll
        for (int m = 0; m < E / R; ++m) {
            C* b = v + m * R * NC;
            if constexpr (LNS > 0) {
                const int k = (c.jt + m * TF) & (NS - 1);
#pragma unroll
                for (int r = 1; r < R; ++r) {
                    const int idx = TWOFF + (r - 1) * NS + k;
                    if constexpr (sizeof(T) == 4) {
                        // FP32 twiddle as hi + lo pairs, applied by one FMA chain per
                        // component: a single rounded twiddle has |w| != 1 by ~3e-8 and
                        // the FFT would shrink or grow the norm coherently every step
                        const float4 w4 = __ldg(reinterpret_cast<const float4*>(a.tw) + idx);
                        const float sh = DIR > 0 ? -w4.y : w4.y, sl = DIR > 0 ? -w4.w : w4.w;
#pragma unroll
                        for (int q = 0; q < NC; ++q) {
                            const C x = b[r * NC + q];
                            const float re = fmaf(x.x, w4.x, fmaf(-x.y, sh, fmaf(x.x, w4.z, -x.y * sl)));
                            const float im = fmaf(x.x, sh, fmaf(x.y, w4.x, fmaf(x.x, sl, x.y * w4.z)));
                            b[r * NC + q] = mk<C>(re, im);
                        }
                    } else if constexpr (DWF) {
                        // double-word twiddle (c_hi, s_hi, c_lo, s_lo), unit modulus far
                        // below the double-word rounding unit; the products stay
                        // unnormalised into this stage's butterfly, whose first level adds
                        // their high parts exactly and renormalises
                        const float4 w4 = __ldg(reinterpret_cast<const float4*>(a.tw) + idx);
                        const DWC w = DWC{DW{w4.x, w4.z}, DIR > 0 ? DW{-w4.y, -w4.w} : DW{w4.y, w4.w}};
#pragma unroll
                        for (int q = 0; q < NC; ++q) b[r * NC + q] = dwc_mul_part(b[r * NC + q], w);
                    } else {
                        C w = __ldg(reinterpret_cast<const C*>(a.tw) + idx);
                        if (DIR > 0) w.y = -w.y;
#pragma unroll
                        for (int q = 0; q < NC; ++q) b[r * NC + q] = cmul(b[r * NC + q], w);
                    }
                }
            }
#pragma unroll
            for (int q = 0; q < NC; ++q) dftR<R, DIR, NC>(b + q);
        }
    }

    // shared-memory unit of (plane p, swizzled index sw) within a buffer:
    //   x axis: bb NPL N + p N + sw = (bb NPL N ^ sw) + p N
    //   y axis: (p N + sw) BATCH + bb = ((sw << log BATCH) ^ bb) + p N BATCH
    static constexpr int LOGB = clog2(BATCH);
    static constexpr int PSTRIDE = AXIS == AXIS_X ? N : N * BATCH;
    KD_DI static int fold(const Ctx& c) { return AXIS == AXIS_X ? c.bb * NPL * N : c.bb; }
    __host__ __device__ static constexpr int lin(int sw) { return AXIS == AXIS_X ? sw : sw << LOGB; }

    // shared-memory exchange XI (0, 1, ... in kernel order) from the output layout of a
    // stage (LA = log Ns, LB = log R) to the input layout of a stage with radix 2^LRN.
    // Consecutive exchanges alternate between two buffers when they fit (one barrier).
    template <int LA, int LB, int LRN, int XI> KD_DI static void exchange(const Ctx& c, C* v) {
        constexpr int R = 1 << LB;
        constexpr int RN = 1 << LRN;
        constexpr int G = Cf::LOGG;
        constexpr int BUF = Cf::DB ? (XI & 1) * Cf::BUF_UNITS : 0;
        U* sm = c.sm + BUF;
        // per-thread bases; j = jt + m TF = jt ^ (m TF) and both maps are XOR-linear
        const int wb = fold(c) ^ lin(swz<LA, LB, G>(expand<LA, LB>(c.jt)));
        const int rb = fold(c) ^ lin(swz<LA, LB, G>(c.jt));
#pragma unroll
        for (int m = 0; m < E / R; ++m)
#pragma unroll
            for (int r = 0; r < R; ++r) {
                const int k = lin(swz<LA, LB, G>(expand<LA, LB>(m * TF)) ^ (r << LA));
#pragma unroll
                for (int p = 0; p < NPL; ++p) sm[(wb ^ k) + p * PSTRIDE] = Unit<T>::pack(v + (m * R + r) * NC + p * CPP);
            }
        block_sync(c);
#pragma unroll
        for (int m = 0; m < E / RN; ++m)
#pragma unroll
            for (int r = 0; r < RN; ++r) {
                const int k = lin(swz<LA, LB, G>((m * TF) | (r << (LOGN - LRN))));
#pragma unroll
                for (int p = 0; p < NPL; ++p) Unit<T>::unpack(sm[(rb ^ k) + p * PSTRIDE], v + (m * RN + r) * NC + p * CPP);
            }
        if constexpr (!Cf::DB) block_sync(c);
    }

    // FFT with stages in plan order (REV = false) or reversed plan order (REV = true)
    template <int DIR, bool REV, int XB, int S> KD_DI static void fft(const SweepArgs& a, const Ctx& c, C* v) {
        if constexpr (S < NST) {
            constexpr int PS = REV ? NST - 1 - S : S;              // plan index of this stage
            constexpr int LR = plan_logr(LOGN, Cf::LOGE, PS);
            constexpr int LNS = REV ? LOGN - plan_logns(LOGN, Cf::LOGE, PS + 1)
                                    : plan_logns(LOGN, Cf::LOGE, PS);
            stage<DIR, LR, LNS, tw_offset(LOGN, Cf::LOGE, REV, S)>(a, c, v);
            if constexpr (S + 1 < NST) {
                constexpr int PN = REV ? NST - 2 - S : S + 1;
                exchange<LNS, LR, plan_logr(LOGN, Cf::LOGE, PN), XB + S>(c, v);
                fft<DIR, REV, XB, S + 1>(a, c, v);
            }
        }
    }

    // --------------------------------------------------------- pointwise ops -------
    // cos(theta) - 1 and sin(theta)/theta as Taylor series in theta^2 (theta < 1/4):
    // truncation below 1e-13 (FP32 terms) and 1e-20 (FP64 terms), so the factor
    // (1 + c1) + i s alpha.a stays unitary far below the rounding unit
    KD_DI static void small_rotation(T th2, T* c1, T* sinc) {
        if constexpr (sizeof(T) == 4) {
            *c1 = th2 * (-0.5f + th2 * (1.0f / 24 + th2 * (-1.0f / 720 + th2 * (1.0f / 40320))));
            *sinc = 1.0f + th2 * (-1.0f / 6 + th2 * (1.0f / 120 + th2 * (-1.0f / 5040 + th2 * (1.0f / 362880))));
        } else {
            *c1 = th2 * (-0.5 + th2 * (1.0 / 24 + th2 * (-1.0 / 720 + th2 * (1.0 / 40320 +
                  th2 * (-1.0 / 3628800 + th2 * (1.0 / 479001600))))));
            *sinc = 1.0 + th2 * (-1.0 / 6 + th2 * (1.0 / 120 + th2 * (-1.0 / 5040 + th2 * (1.0 / 362880 +
                    th2 * (-1.0 / 39916800 + th2 * (1.0 / 6227020800.0))))));
        }
    }
    KD_DI static T fexp(T x) {
        if constexpr (sizeof(T) == 4) return __expf(x); else return exp(x);
    }
    KD_DI static void fsincos(T x, T* s, T* c) {
        if constexpr (sizeof(T) == 4) __sincosf(x, s, c); else sincos(x, s, c);
    }

    // potential factor exp(-i tau V/hbar), V = -m c^2 alpha.a, on registers in the op
    // layout (element index j + r N/R_op is the x index of the row).  The standing wave
    // sum over d = +-1 of Eqs. (Equation_of_Gaussian_beam) is taken in product form:
    //   a_y = -2 s(t) G cos(Theta),  a_x = 4 eps s(t) (y/w) G sin(Theta + zeta),
    //   G = (w0/w) exp(-y^2/w^2),  Theta = -k x + zeta - x y^2/(x_R w^2),  zeta = atan(x/x_R),
    // with s(t) = a0 f(t) sin(omega t + phase0) from the FP64 per-step table and the
    // x-dependent parts from the FP64 per-x table.  FP32 uses the SFU exp/sincos on
    // |Theta| <= pi + 1 (absolute error ~5e-7 of the field, no effect on unitarity).
    // per-row scalars of the potential step: y of the row in the moving box and the
    // standing wave's time factor, read (device clock, then the step's scalars) right
    // after the grid-dependency wait so that the two dependent loads overlap the row load
    struct RowField {
        T y, st;
    };
    KD_DI static RowField row_field(const SweepArgs& a, const Ctx& c) {
        RowField f{};
        if (AXIS != AXIS_X || a.op != OP_POTENTIAL || a.kind == 0) return f;
        const Clock ck = *a.clock;
        const StepScalars* ssp = a.steps + ((ck.step - ck.base) + c.n_local);
        if constexpr (DWF) {
            f.y = dw_from_double(ssp->ybase + (double)c.line * a.dy);
            f.st = dw_from_double(ssp->s);
        } else if constexpr (sizeof(T) == 4) {
            f.y = ssp->ybase_f + (float)c.line * a.dy_f;
            f.st = ssp->s_f;
        } else {
            f.y = ssp->ybase + (double)c.line * a.dy;
            f.st = ssp->s;
        }
        return f;
    }

    KD_DI static void op_potential(const SweepArgs& a, const Ctx& c, C* v, const RowField rf) {
        if constexpr (DWF) op_potential_dw(a, c, v, rf);
        else op_potential_std(a, c, v, rf);
    }

    // the double-word potential step: the field of the standing wave as in op_potential_std
    // with every quantity a double-word and exp, sin, cos of kd_dw.cuh (relative error
    // ~1e-14 of the field, so that the factor is exact to the double-word rounding unit
    // over thousands of steps); table a.xtab holds per column x two double-word 4-vectors
    // (Theta0, x/(x_R w^2), w0/w, 1/w^2) and (1/w, cos zeta, sin zeta, cos k x) as four
    // float4 [2][nx][2]
    KD_DI static void op_potential_dw(const SweepArgs& a, const Ctx& c, C* v, const RowField rf) {
        if constexpr (DWF) {
            if (a.kind == 0) return;
            constexpr int R = 1 << LR_OP;
            const DW y = rf.y, st = rf.st;
            const DW y2 = dw_mul(y, y);
            const DW kap = dw_from_double(a.kappa), e4 = dw_from_double(a.eps4);
            if constexpr (!Cf::SHARE) {
                // pairs in separate CTAs (lines of more than 256 threads): every thread
                // evaluates the factors of all its points
#pragma unroll
                for (int m = 0; m < E / R; ++m)
#pragma unroll
                    for (int r = 0; r < R; ++r) {
                        const int x = c.jt + m * TF + r * (N / R);
                        const DWFactor f = dw_potential_factor(a.xtab, a.dwconst, a.nx, x, a.kind,
                                                               a.longitudinal, y, y2, st, kap, e4);
                        apply_potential_dw(c, v + (m * R + r) * NC, f.c1, f.say, f.sax);
                    }
                return;
            }
            // the two pairs' threads own the same points: each evaluates the factors of the
            // points of parity c.pair into shared memory, and both read all of them back
            constexpr int SLOT = Cf::DB ? ((NST - 1) & 1) * Cf::BUF_UNITS : 0;
            float4* fsh = reinterpret_cast<float4*>(c.sm + SLOT) + 2 * (c.bb % BATCH) * N;
#pragma unroll
            for (int m = 0; m < E / R; ++m)
#pragma unroll
                for (int r = 0; r < R; ++r) {
                    if (((m * R + r) & 1) != c.pair) continue;
                    const int x = c.jt + m * TF + r * (N / R);
                    const DWFactor f = dw_potential_factor(a.xtab, a.dwconst, a.nx, x, a.kind, a.longitudinal,
                                                           y, y2, st, kap, e4);
                    if (c.valid) {
                        fsh[2 * x] = make_float4(f.c1.h, f.c1.l, f.say.h, f.say.l);
                        fsh[2 * x + 1] = make_float4(f.sax.h, f.sax.l, 0.0f, 0.0f);
                    }
                }
            block_sync(c);
#pragma unroll
            for (int m = 0; m < E / R; ++m)
#pragma unroll
                for (int r = 0; r < R; ++r) {
                    const int x = c.jt + m * TF + r * (N / R);
                    const float4 f0 = c.valid ? fsh[2 * x] : make_float4(0.f, 0.f, 0.f, 0.f);
                    const float4 f1 = c.valid ? fsh[2 * x + 1] : make_float4(0.f, 0.f, 0.f, 0.f);
                    apply_potential_dw(c, v + (m * R + r) * NC, DW{f0.x, f0.y}, DW{f0.z, f0.w}, DW{f1.x, f1.y});
                }
            if constexpr (!Cf::DB) block_sync(c);
        }
    }

    // (1 + c1) + i (s a).alpha on this thread's pair at one point, double-word: say = s a_y
    // (negated for pair 1), sax = s a_x
    KD_DI static void apply_potential_dw(const Ctx& c, C* e, DW c1, DW say0, DW sax) {
        if constexpr (DWF) {
            const DW say = c.pair == 0 ? say0 : dw_neg(say0);
            const C u = e[0], l = e[1];
            const C q1 = C{say, sax}, q2 = C{dw_neg(say), sax};
            const C du = dwc_add(dwc_mul_r(u, c1), dwc_mul(l, q1));
            const C dl = dwc_add(dwc_mul_r(l, c1), dwc_mul(u, q2));
            e[0] = dwc_add(u, du);
            e[1] = dwc_add(l, dl);
        }
    }

    KD_DI static void op_potential_std(const SweepArgs& a, const Ctx& c, C* v, const RowField rf) {
        if (a.kind == 0) return;
        constexpr int R = 1 << LR_OP;
        using T4 = typename std::conditional<sizeof(T) == 4, float4, double4>::type;
        const T y = rf.y, st = rf.st;
        T kap, e4;
        if constexpr (sizeof(T) == 4) {
            kap = a.kappa_f;
            e4 = a.eps4_f;
        } else {
            kap = a.kappa;
            e4 = a.eps4;
        }
        const T y2 = y * y;
        const T kap2 = kap * kap;
        const T4* xt = reinterpret_cast<const T4*>(a.xtab);   // [2][nx] vectors
        const int nx = a.nx;
        // field sharing: this thread evaluates the points e = m R + r of parity c.pair, and
        // both pairs' threads read all factors (cos theta - 1, s a_y, s a_x) back from
        // shared memory
        float4* fsh = nullptr;
        if constexpr (Cf::SHARE) {
            constexpr int SLOT = Cf::DB ? ((NST - 1) & 1) * Cf::BUF_UNITS : 0;
            fsh = reinterpret_cast<float4*>(c.sm + SLOT) + (c.bb % BATCH) * N;
        }
#pragma unroll
        for (int m = 0; m < E / R; ++m)
#pragma unroll
            for (int r = 0; r < R; ++r) {
                const int x = c.jt + m * TF + r * (N / R);
                if constexpr (Cf::SHARE) {
                    if (((m * R + r) & 1) != c.pair) continue;
                }
                const T4 t1 = xt[nx + x];        // (1/w, cos zeta, sin zeta, cos k x)
                T ax = T(0), ay;
                if (a.kind == 1) {
                    ay = T(-2) * st * t1.w;
                } else {
                    const T4 t0 = xt[x];         // (Theta0, x/(x_R w^2), w0/w, 1/w^2)
                    const T G = t0.z * fexp(-y2 * t0.w);
                    T th = t0.x - t0.y * y2;
                    if constexpr (sizeof(T) == 4) th -= 6.283185307f * rintf(th * 0.159154943f);
                    T sn, cs;
                    fsincos(th, &sn, &cs);
                    const T sg = st * G;
                    ay = T(-2) * sg * cs;
                    if (a.longitudinal) ax = e4 * sg * (y * t1.x) * (sn * t1.y + cs * t1.z);
                }
                const T a2 = ax * ax + ay * ay;
                const T th2 = kap2 * a2;
                T c1, s;   // cos(theta) - 1 and sin(theta)/|a|, theta = kappa |a|
                if (th2 < T(0.0625)) {
                    T sinc;
                    small_rotation(th2, &c1, &sinc);
                    s = kap * sinc;
                } else {
                    const T amag = sqrt(a2);
                    T sh, ch;
                    sincos_(T(0.5) * kap * amag, &sh, &ch);
                    c1 = T(-2) * sh * sh;
                    s = T(2) * sh * ch / amag;
                }
                if constexpr (Cf::SHARE) {
                    if (c.valid) fsh[x] = make_float4(c1, s * ay, s * ax, 0.0f);
                } else {
                    apply_potential(c, v + (m * R + r) * NC, c1, s * ay, s * ax);
                }
            }
        if constexpr (Cf::SHARE) {
            block_sync(c);
#pragma unroll
            for (int m = 0; m < E / R; ++m)
#pragma unroll
                for (int r = 0; r < R; ++r) {
                    const int x = c.jt + m * TF + r * (N / R);
                    const float4 f = c.valid ? fsh[x] : make_float4(0.f, 0.f, 0.f, 0.f);
                    apply_potential(c, v + (m * R + r) * NC, f.x, f.y, f.z);
                }
            // single buffer: the next exchange writes over the factors
            if constexpr (!Cf::DB) block_sync(c);
        }
    }

    // (1 + c1) + i (s a).alpha on the pairs of one point: say = s a_y, sax = s a_x (pair 1's
    // generator has a_y negated)
    KD_DI static void apply_potential(const Ctx& c, C* e, T c1, T say, T sax) {
#pragma unroll
        for (int q = 0; q < NC / 2; ++q) {
            const int pr = NC == 4 ? q : c.pair;
            const T sy = pr == 0 ? say : -say;
            const C u = e[2 * q], l = e[2 * q + 1];
            const C q1 = mk<C>(sy, sax);
            const C q2 = mk<C>(-sy, sax);
            const C du = cadd(mk<C>(c1 * u.x, c1 * u.y), cmul(q1, l));
            const C dl = cadd(mk<C>(c1 * l.x, c1 * l.y), cmul(q2, u));
            e[2 * q] = cadd(u, du);
            e[2 * q + 1] = cadd(l, dl);
        }
    }

    // kinetic factor e^{i phi} [C - i S H0(pi)] / P on registers; element index is k_y,
    // the line is k_x.  Stored as small numbers so that no constant next to 1 is rounded:
    // per point a = (C - 1)/P and b = c S/P (chosen so that the factor built from the
    // same rounded pi and m c as below is unitary to ~1e-11), per row f = e^{i phi} - 1
    // (unit modulus of 1 + f to ~1e-12).  Applied as psi/P + a psi - i b (H0/c) psi, then
    // times 1 + f; each result is a rounding around psi itself, which carries no bias.
    // per-point kinetic table entries of this thread (op layout), loaded at kernel start
    // so that their L2 latency overlaps the first FFT
    KD_DI static void load_ktab(const SweepArgs& a, const Ctx& c, C* kab) {
        constexpr int R = 1 << LR_OP;
        const C* kt = reinterpret_cast<const C*>(a.ktab);
#pragma unroll
        for (int m = 0; m < E / R; ++m)
#pragma unroll
            for (int r = 0; r < R; ++r) {
                const int ky = c.jt + m * TF + r * (N / R);
                if constexpr (DWF) {
                    const float4 q = c.valid ? __ldcg(reinterpret_cast<const float4*>(a.ktab) + (long long)ky * a.nx + c.line)
                                             : make_float4(0.f, 0.f, 0.f, 0.f);
                    kab[m * R + r] = DWC{DW{q.x, q.y}, DW{q.z, q.w}};
                } else {
                    kab[m * R + r] = c.valid ? __ldcg(kt + (long long)ky * a.nx + c.line) : mk<C>(T(0), T(0));
                }
            }
    }

    KD_DI static void op_kinetic(const SweepArgs& a, const Ctx& c, C* v, const C* kab) {
        if constexpr (DWF) op_kinetic_dw(a, c, v, kab);
        else op_kinetic_std(a, c, v, kab);
    }

    // the double-word kinetic step, the same factor as op_kinetic_std: tables a.kxtab
    // [nx] double-word pi_x (float2), a.kytab [ny][2] float4 (pi_y, cos phi - 1 | sin phi),
    // a.ktab [ny][nx] float4 ((C - 1)/P, c S/P)
    KD_DI static void op_kinetic_dw(const SweepArgs& a, const Ctx& c, C* v, const C* kab) {
        if constexpr (DWF) {
            constexpr int R = 1 << LR_OP;
            const float2 px = __ldg(reinterpret_cast<const float2*>(a.kxtab) + c.line);
            const DW pix = DW{px.x, px.y};
            const DW mc = dw_from_double(a.mc);
            const float invP = (float)a.invP;   // a power of two: exact
            const float4* kyt = reinterpret_cast<const float4*>(a.kytab);
#pragma unroll
            for (int m = 0; m < E / R; ++m)
#pragma unroll
                for (int r = 0; r < R; ++r) {
                    const int ky = c.jt + m * TF + r * (N / R);
                    const C ab = kab[m * R + r];
                    const float4 y0 = __ldg(kyt + 2 * ky), y1 = __ldg(kyt + 2 * ky + 1);
                    const DW fx = DW{y0.z, y0.w}, fy = DW{y1.x, y1.y};
                    C* e = v + (m * R + r) * NC;
#pragma unroll
                    for (int q = 0; q < NC / 2; ++q) {
                        const int pr = NC == 4 ? q : c.pair;
                        const DW piy = pr == 0 ? DW{y0.x, y0.y} : DW{-y0.x, -y0.y};
                        const C u = e[2 * q], l = e[2 * q + 1];
                        // G = H0/c on the pair: (mc u + (pix - i piy) l, (pix + i piy) u - mc l)
                        const C hu = C{dw_add(dw_dot2(mc, u.x, pix, l.x), dw_mul(piy, l.y)),
                                       dw_sub(dw_dot2(mc, u.y, pix, l.y), dw_mul(piy, l.x))};
                        const C hl = C{dw_sub(dw_dot2(pix, u.x, piy, dw_neg(u.y)), dw_mul(mc, l.x)),
                                       dw_sub(dw_dot2(pix, u.y, piy, u.x), dw_mul(mc, l.y))};
                        // u/P + a u - i b hu
                        const C u1 = C{dw_add(dw_scale(u.x, invP), dw_dot2(ab.x, u.x, ab.y, hu.y)),
                                       dw_add(dw_scale(u.y, invP), dw_dot2(ab.x, u.y, dw_neg(ab.y), hu.x))};
                        const C l1 = C{dw_add(dw_scale(l.x, invP), dw_dot2(ab.x, l.x, ab.y, hl.y)),
                                       dw_add(dw_scale(l.y, invP), dw_dot2(ab.x, l.y, dw_neg(ab.y), hl.x))};
                        // times 1 + f (frame translation phase)
                        e[2 * q] = C{dw_add(u1.x, dw_dot2(fx, u1.x, dw_neg(fy), u1.y)),
                                     dw_add(u1.y, dw_dot2(fx, u1.y, fy, u1.x))};
                        e[2 * q + 1] = C{dw_add(l1.x, dw_dot2(fx, l1.x, dw_neg(fy), l1.y)),
                                         dw_add(l1.y, dw_dot2(fx, l1.y, fy, l1.x))};
                    }
                }
        }
    }

    KD_DI static void op_kinetic_std(const SweepArgs& a, const Ctx& c, C* v, const C* kab) {
        constexpr int R = 1 << LR_OP;
        const T pix = __ldg(reinterpret_cast<const T*>(a.kxtab) + c.line);
        T mc, invP;   // invP = 1/P is exact (power of two)
        if constexpr (sizeof(T) == 4) { mc = a.mc_f; invP = a.invP_f; }
        else { mc = a.mc; invP = a.invP; }
        using T4 = typename std::conditional<sizeof(T) == 4, float4, double4>::type;
        const T4* kyt = reinterpret_cast<const T4*>(a.kytab);
#pragma unroll
        for (int m = 0; m < E / R; ++m)
#pragma unroll
            for (int r = 0; r < R; ++r) {
                const int ky = c.jt + m * TF + r * (N / R);
                const C ab = kab[m * R + r];
                const T4 yv = kyt[ky];                   // (pi_y, cos phi - 1, sin phi, 0)
                C* e = v + (m * R + r) * NC;
#pragma unroll
                for (int q = 0; q < NC / 2; ++q) {
                    const int pr = NC == 4 ? q : c.pair;
                    const T piy = pr == 0 ? yv.x : -yv.x;
                    const C u = e[2 * q], l = e[2 * q + 1];
                    // G = H0/c on the pair: (mc u + (pix - i piy) l, (pix + i piy) u - mc l)
                    const C hu = mk<C>(mc * u.x + pix * l.x + piy * l.y, mc * u.y + pix * l.y - piy * l.x);
                    const C hl = mk<C>(pix * u.x - piy * u.y - mc * l.x, pix * u.y + piy * u.x - mc * l.y);
                    // u/P + a u - i b hu
                    const C u1 = mk<C>(u.x * invP + (ab.x * u.x + ab.y * hu.y), u.y * invP + (ab.x * u.y - ab.y * hu.x));
                    const C l1 = mk<C>(l.x * invP + (ab.x * l.x + ab.y * hl.y), l.y * invP + (ab.x * l.y - ab.y * hl.x));
                    // times 1 + f (frame translation phase)
                    e[2 * q] = mk<C>(u1.x + (yv.y * u1.x - yv.z * u1.y), u1.y + (yv.y * u1.y + yv.z * u1.x));
                    e[2 * q + 1] = mk<C>(l1.x + (yv.y * l1.x - yv.z * l1.y), l1.y + (yv.y * l1.y + yv.z * l1.x));
                }
            }
    }

    KD_DI static void sincos_(float x, float* s, float* c) { sincosf(x, s, c); }
    KD_DI static void sincos_(double x, double* s, double* c) { sincos(x, s, c); }

    KD_DI static void run(const SweepArgs& a) {
        extern __shared__ __align__(16) unsigned char smem_raw[];
        run_block<true>(a, (int)blockIdx.x, (int)threadIdx.x, smem_raw, a.n_local, 0);
    }

    // One launch block `blk` of the sweep, executed by the THREADS threads tid = 0..THREADS-1
    // with `smem` (SMEM_BYTES) as its shared memory.  PDL: a standalone launch waits for the
    // previous grid here; the persistent batch kernel (kd_persist.cu) runs blocks as work
    // items after its own dependency wait (every thread of the CTA reaches the same
    // barriers: items of one kind run side by side with the same instantiation).
    template <bool PDL>
    KD_DI static void run_block(const SweepArgs& a, int blk, int tid, unsigned char* smem, int n_local, int bar) {
        Ctx c;
        c.n_local = n_local;
        c.bar = bar;
        if (AXIS == AXIS_X) { c.bb = tid / TF; c.jt = tid % TF; }
        else { c.bb = tid % BATCH; c.jt = tid / BATCH; }
        // the pair index varies fastest so both pairs of a line tile run together; with
        // field sharing both pairs are in the CTA (c.bb then counts PCTA x BATCH lines)
        if constexpr (Cf::SHARE) c.pair = c.bb / BATCH;
        else c.pair = NC == 2 ? blk % Cf::NPAIRS : 0;
        c.line = (blk / Cf::NPAIRS) * BATCH + c.bb % BATCH;
        c.valid = c.line < (AXIS == AXIS_X ? a.ny : a.nx);
        c.sm = reinterpret_cast<U*>(smem);
        C v[E * NC];
        // programmatic dependent launch: everything above ran while the previous kernel
        // in the stream was still finishing; its results are visible after this wait
        // (a hardware-managed wait for the prerequisite grid, not a spin loop)
        if constexpr (PDL) asm volatile("griddepcontrol.wait;" ::: "memory");
        const RowField rf = row_field(a, c);
        load<LR_LOAD>(a, c, v);
        // the next kernel may start its own prologue as our CTAs retire
        if constexpr (PDL) asm volatile("griddepcontrol.launch_dependents;");
        if constexpr (AXIS == AXIS_Y) {
            C kab[E];
            if (a.op == OP_KINETIC) load_ktab(a, c, kab);
            if constexpr (HAS1) fft<DIR1, false, 0, 0>(a, c, v);
            if (a.op == OP_KINETIC) op_kinetic(a, c, v, kab);
        } else {
            if constexpr (HAS1) fft<DIR1, false, 0, 0>(a, c, v);
            if (a.op == OP_POTENTIAL) op_potential(a, c, v, rf);
        }
        // with field sharing the factor trade takes exchange slot NST - 1, so FFT2 starts at NST
        if constexpr (HAS2) fft<DIR2, true, Cf::SHARE ? NST : (HAS1 ? NST - 1 : 0), 0>(a, c, v);
        store<LR_STORE>(a, c, v);
    }
};

template <typename T, int LOGN, int AXIS, int SHAPE, int V>
__global__ void __launch_bounds__(Cfg<T, LOGN, AXIS, V>::THREADS, Cfg<T, LOGN, AXIS, V>::MINBLK)
sweep_kernel(const SweepArgs a) {
    Sweep<T, LOGN, AXIS, SHAPE, V>::run(a);
}

template <typename T, int LOGN, int AXIS, int SHAPE, int V>
cudaError_t launch_one(const SweepArgs& a, cudaStream_t s) {
    using Cf = Cfg<T, LOGN, AXIS, V>;
    static bool attr_done = false;
    auto k = sweep_kernel<T, LOGN, AXIS, SHAPE, V>;
    if (!attr_done) {
        cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                              Cf::SMEM_BYTES);
        if (e != cudaSuccess) return e;
        attr_done = true;
    }
    const int lines = AXIS == AXIS_X ? a.ny : a.nx;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(((lines + Cf::BATCH - 1) / Cf::BATCH) * Cf::NPAIRS);
    cfg.blockDim = dim3(Cf::THREADS);
    cfg.dynamicSmemBytes = Cf::SMEM_BYTES;
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, k, a);
}

// Fills the stage-major twiddle table of an N = 2^LOGN sweep with 2^LOGE elements per
// thread in FP64 (sincospi): FP32 entries are float4 (c_hi, s_hi, c_lo, s_lo), FP64
// entries double2 (c, s).
template <typename T, int LOGN, int LOGE>
__global__ void twiddle_kernel(void* out) {
    constexpr int NST = plan_nst(LOGN, LOGE);
    const int total = tw_total(LOGN, LOGE);
    for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < total; e += gridDim.x * blockDim.x) {
        // find the (order, stage) segment holding entry e and the index within it
        int idx = e, lns = 0, lr = 0;
        bool found = false;
        for (int o = 0; o < 2 && !found; ++o)
            for (int S = 0; S < NST && !found; ++S) {
                const int n = stage_tw_entries(LOGN, LOGE, o == 1, S);
                if (idx < n) {
                    lns = stage_lns(LOGN, LOGE, o == 1, S);
                    lr = stage_lr(LOGN, LOGE, o == 1, S);
                    found = true;
                } else {
                    idx -= n;
                }
            }
        const int ns = 1 << lns;
        const int r = idx / ns + 1, k = idx % ns;
        double sn, cs;
        sincospi(2.0 * (double)(r * k) / (double)(ns << lr), &sn, &cs);
        sn = -sn;
        if constexpr (std::is_same<T, DW>::value) {
            // double-word entries (c_hi, s_hi, c_lo, s_lo): among the lo parts within 3 FP32
            // steps of the rounded residuals, the pair whose represented (C, S) has
            // C^2 + S^2 closest to 1 (evaluated exactly with FP64 TwoProd/TwoSum), with a
            // small weight on the distance to (cos, sin): a twiddle of modulus 1 + d would
            // change the norm by 2 d at every product, coherently over the steps of a run
            const float ch = (float)cs, sh = (float)sn;
            const float cl0 = (float)(cs - (double)ch), sl0 = (float)(sn - (double)sh);
            float bc = cl0, bs = sl0;
            double best = 1e300;
            float ci = cl0;
            for (int q = 0; q < 3; ++q) ci = nextafterf(ci, -INFINITY);
            for (int i = 0; i < 7; ++i, ci = nextafterf(ci, INFINITY)) {
                float si = sl0;
                for (int q = 0; q < 3; ++q) si = nextafterf(si, -INFINITY);
                for (int j = 0; j < 7; ++j, si = nextafterf(si, INFINITY)) {
                    const double C = (double)ch + (double)ci, S = (double)sh + (double)si;
                    const double pc = C * C, ec = fma(C, C, -pc);
                    const double ps = S * S, es = fma(S, S, -ps);
                    const double hi = pc + ps, bb = hi - pc;
                    const double lo = (pc - (hi - bb)) + (ps - bb);
                    const double d = ((hi - 1.0) + lo) + (ec + es);
                    const double g = fabs(d) + 0.05 * (fabs(C - cs) + fabs(S - sn));
                    if (g < best) { best = g; bc = ci; bs = si; }
                }
            }
            reinterpret_cast<float4*>(out)[e] = make_float4(ch, sh, bc, bs);
        } else if constexpr (sizeof(T) == 4) {
            const float ch = (float)cs, sh = (float)sn;
            reinterpret_cast<float4*>(out)[e] = make_float4(ch, sh, (float)(cs - (double)ch), (float)(sn - (double)sh));
        } else {
            reinterpret_cast<double2*>(out)[e] = make_double2(cs, sn);
        }
    }
}

template <typename T, int LOGN, int LOGE> cudaError_t build_tw(void* out, int* entries, cudaStream_t s) {
    constexpr int LE = LOGE < LOGN ? LOGE : LOGN;
    *entries = tw_total(LOGN, LE);
    if (*entries > 0) twiddle_kernel<T, LOGN, LE><<<(*entries + 255) / 256, 256, 0, s>>>(out);
    return cudaGetLastError();
}

template <typename T, int LOGN> cudaError_t build_tw_e(int loge, void* out, int* entries, cudaStream_t s) {
    if (loge == 2) return build_tw<T, LOGN, 2>(out, entries, s);
    if (loge == 3) return build_tw<T, LOGN, 3>(out, entries, s);
    return cudaErrorInvalidValue;
}

template <typename T> cudaError_t build_twiddles(int logn, int loge, void* out, int* entries, cudaStream_t s) {
    switch (logn) {
        case 2: return build_tw_e<T, 2>(loge, out, entries, s);
        case 3: return build_tw_e<T, 3>(loge, out, entries, s);
        case 4: return build_tw_e<T, 4>(loge, out, entries, s);
        case 5: return build_tw_e<T, 5>(loge, out, entries, s);
        case 6: return build_tw_e<T, 6>(loge, out, entries, s);
        case 7: return build_tw_e<T, 7>(loge, out, entries, s);
        case 8: return build_tw_e<T, 8>(loge, out, entries, s);
        case 9: return build_tw_e<T, 9>(loge, out, entries, s);
        case 10: return build_tw_e<T, 10>(loge, out, entries, s);
        case 11: return build_tw_e<T, 11>(loge, out, entries, s);
        case 12: return build_tw_e<T, 12>(loge, out, entries, s);
        default: return cudaErrorInvalidValue;
    }
}

template <typename T, int AXIS, int SHAPE, int V>
cudaError_t launch_logn(int logn, const SweepArgs& a, cudaStream_t s) {
    switch (logn) {
        case 2: return launch_one<T, 2, AXIS, SHAPE, V>(a, s);
        case 3: return launch_one<T, 3, AXIS, SHAPE, V>(a, s);
        case 4: return launch_one<T, 4, AXIS, SHAPE, V>(a, s);
        case 5: return launch_one<T, 5, AXIS, SHAPE, V>(a, s);
        case 6: return launch_one<T, 6, AXIS, SHAPE, V>(a, s);
        case 7: return launch_one<T, 7, AXIS, SHAPE, V>(a, s);
        case 8: return launch_one<T, 8, AXIS, SHAPE, V>(a, s);
        case 9: return launch_one<T, 9, AXIS, SHAPE, V>(a, s);
        case 10: return launch_one<T, 10, AXIS, SHAPE, V>(a, s);
        case 11: return launch_one<T, 11, AXIS, SHAPE, V>(a, s);
        case 12: return launch_one<T, 12, AXIS, SHAPE, V>(a, s);
        default: return cudaErrorInvalidValue;
    }
}

template <typename T, int V>
cudaError_t launch_sweep(int axis, int shape, int logn, const SweepArgs& a, cudaStream_t s) {
    if (axis == AXIS_X) {
        if (shape == SHAPE_F1F2) return launch_logn<T, AXIS_X, SHAPE_F1F2, V>(logn, a, s);
        if (shape == SHAPE_F1) return launch_logn<T, AXIS_X, SHAPE_F1, V>(logn, a, s);
        if (shape == SHAPE_F2) return launch_logn<T, AXIS_X, SHAPE_F2, V>(logn, a, s);
    } else {
        if (shape == SHAPE_F1F2) return launch_logn<T, AXIS_Y, SHAPE_F1F2, V>(logn, a, s);
        if (shape == SHAPE_F1) return launch_logn<T, AXIS_Y, SHAPE_F1, V>(logn, a, s);
        if (shape == SHAPE_F2) return launch_logn<T, AXIS_Y, SHAPE_F2, V>(logn, a, s);
    }
    return cudaErrorInvalidValue;
}

}  // namespace kd
