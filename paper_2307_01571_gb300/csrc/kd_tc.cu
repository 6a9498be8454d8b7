// kd_tc.cu -- precision form of the fused sweeps: the 1024-point FFTs of the split-operator
// step (Sec. II.D of arXiv 2307.01571) evaluated as dense 32-point DFT matrix products on
// the tensor cores (tcgen05, FP16 operands split hi + lo, FP32 accumulation in TMEM).
//
// A sweep over lines of N = 1024 = 32 x 32 points runs, per line, the four-step FFT:
//   S1  32-point DFTs over q of x[p + 32 q] (one vector per p),
//   T1  twiddle w_N^(p k2),
//   S2  32-point DFTs over p (one vector per k2): X[k2 + 32 k1],
// then the pointwise factor (potential on the x axis, kinetic on the y axis) on
// X[k2 + 32 k1] in place, then the second FFT with the roles of the two factors swapped
// (S3 over k1 of each k2-vector, T2, S4), which leaves Y[c2 + 32 c1] in the row of c2.
// Every DFT stage is one matrix product D = A B^T per spinor component with
//   A = [128 vectors x 32 complex] (rows = 4 lines x 32 vectors, interleaved re/im),
//   B = the real 64 x 64 form of the 32-point DFT matrix ([[c, -s], [s, c]] blocks),
// M = 128, N = 64, K = 64, issued by one thread as 3 terms x 4 K-steps per component:
//   A_hi B_hi + A_lo B_hi + A_hi B_lo   (hi = fp16(v), lo = fp16(v - hi): ~22 bits).
// The products accumulate in FP32 in tensor memory; two threads share each row (row r =
// TMEM lane r, one thread per half of its columns) and read it back with tcgen05.ld, apply
// the twiddle or the pointwise factor in FP32 on registers and write the next stage's
// operand to shared memory, transposing between S1 and S2 (and S3 and S4) by their
// scattered stores.
//
// FP16 range: values are carried with power-of-two scales (exact) chosen per sweep from
// the state's 2-norm, so that no operand can exceed 2^14 (bounds from the growth of the
// unnormalised DFTs), and the DFT matrix is stored times 2^10 so that its lo parts stay
// normal FP16 numbers.  Operand rounding is ~1e-7 of the line maximum per stage (FP32
// CUDA-core stages: ~6e-8), but the tensor cores' FP32 accumulation truncates, which
// shrinks the norm by ~2e-7 per stage (~7e-7 per Strang step with one axis here).  Only the
// full sweeps (both FFTs) of N = 1024 axes run here; the half sweeps at run ends and other
// axis lengths use the FP32 CUDA-core kernels.
#include <cuda_fp16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include "kd_internal.h"

namespace kd {
namespace tc {

// 256 threads: two per accumulator row (TMEM lane), each handling half of the row's 32
// complex columns in every phase, so that 16 warps per SM hide the latencies
constexpr int N = 1024, L = 32, LC = 4, THREADS = 256, HALF = L / 2;
// A operand tile of one component: 128 rows x 32 complex FP16 in the no-swizzle K-major
// canonical layout (8-row x 16-byte core matrices); LBO = byte step between core matrices
// along K, SBO = byte step between 8-row groups.  The padding (144 instead of 128, 1168
// instead of 1152) makes the transposing 4-byte stores and the 16-byte row stores
// bank-conflict free.
constexpr uint32_t LBO = 144, SBO = 1168, TILE = 16 * SBO;
// B operand: 64 x 64 FP16, dense canonical layout
constexpr uint32_t BLBO = 128, BSBO = 1024, BMAT = 8 * BSBO;
constexpr uint32_t OFF_AHI = 0, OFF_ALO = 2 * TILE, OFF_B = 4 * TILE;
constexpr uint32_t OFF_BAR = OFF_B + 4 * BMAT, OFF_SLOT = OFF_BAR + 8;
constexpr uint32_t SMEM = OFF_SLOT + 8;
// D of the two components, 64 columns each: A_hi B_hi in columns [0, 128), the two small
// cross terms A_lo B_hi + A_hi B_lo in [128, 256), summed in FP32 on the CUDA cores (the
// tensor cores' accumulation truncates; keeping the small terms out of the large
// accumulator removes two thirds of the truncations at full magnitude)
constexpr uint32_t TMEM_COLS = 256;
constexpr float BSCALE_INV = 1.0f / 1024.0f;       // the DFT matrix is stored times 2^10
// instruction descriptor: FP16 A and B (K-major), FP32 D, N = 64, M = 128
constexpr uint32_t IDESC = (1u << 4) | ((uint32_t)(64 >> 3) << 17) | ((uint32_t)(128 >> 4) << 24);
constexpr long long WAIT_LIMIT = 1ll << 20;        // try_wait polls before giving up

static_assert(SMEM <= 110 * 1024, "two CTAs per SM");

__device__ __forceinline__ uint32_t su32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

// shared-memory matrix descriptor (tcgen05): start, LBO, SBO (all >> 4), version 1,
// no swizzle
__device__ __forceinline__ uint64_t sdesc(uint32_t saddr, uint32_t lbo, uint32_t sbo) {
    return (uint64_t)((saddr & 0x3FFFF) >> 4) | ((uint64_t)((lbo >> 4) & 0x3FFF) << 16) |
           ((uint64_t)((sbo >> 4) & 0x3FFF) << 32) | ((uint64_t)1 << 46);
}

__device__ __forceinline__ uint32_t aoff(int r, int col) {   // byte offset of complex (r, col)
    return (uint32_t)(r >> 3) * SBO + (uint32_t)(col >> 2) * LBO + (uint32_t)(r & 7) * 16 + (uint32_t)(col & 3) * 4;
}

__device__ __forceinline__ void mma_f16(uint32_t d, uint64_t a, uint64_t b, uint32_t acc) {
    asm volatile("{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
                 "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}"
                 :: "r"(d), "l"(a), "l"(b), "r"(IDESC), "r"(acc));
}

__device__ __forceinline__ bool mbar_try(uint32_t bar, uint32_t parity) {
    uint32_t ok;
    asm volatile("{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
                 "selp.u32 %0, 1, 0, p;\n\t}" : "=r"(ok) : "r"(bar), "r"(parity) : "memory");
    return ok != 0;
}

// bounded wait for the phase `parity` of the MMA barrier
__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t parity) {
    for (long long it = 0; it < WAIT_LIMIT; ++it)
        if (mbar_try(bar, parity)) return true;
    return false;
}

// 16 FP32 columns of this thread's TMEM lane (row), starting at column `col`
#define KD_TMEM_LD16(taddr, r)                                                                  \
    asm volatile("tcgen05.ld.sync.aligned.32x32b.x16.b32 "                                     \
                 "{%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"             \
                 : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]),      \
                   "=r"(r[6]), "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]),    \
                   "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])                           \
                 : "r"(taddr))

// completes the loads of the two 16-column chunks; the registers pass through the asm so
// that no use of them can be scheduled before the wait
__device__ __forceinline__ void tmem_wait2(uint32_t* u, uint32_t* l) {
    asm volatile("tcgen05.wait::ld.sync.aligned;"
                 : "+r"(u[0]), "+r"(u[1]), "+r"(u[2]), "+r"(u[3]), "+r"(u[4]), "+r"(u[5]), "+r"(u[6]),
                   "+r"(u[7]), "+r"(u[8]), "+r"(u[9]), "+r"(u[10]), "+r"(u[11]), "+r"(u[12]),
                   "+r"(u[13]), "+r"(u[14]), "+r"(u[15]), "+r"(l[0]), "+r"(l[1]), "+r"(l[2]),
                   "+r"(l[3]), "+r"(l[4]), "+r"(l[5]), "+r"(l[6]), "+r"(l[7]), "+r"(l[8]), "+r"(l[9]),
                   "+r"(l[10]), "+r"(l[11]), "+r"(l[12]), "+r"(l[13]), "+r"(l[14]), "+r"(l[15])
                 :: "memory");
}

// (re, im) -> packed FP16 hi and lo parts
__device__ __forceinline__ void split(float re, float im, uint32_t* hi, uint32_t* lo) {
    const __half2 h = __floats2half2_rn(re, im);
    const float2 hf = __half22float2(h);
    const __half2 l = __floats2half2_rn(re - hf.x, im - hf.y);
    *hi = *reinterpret_cast<const uint32_t*>(&h);
    *lo = *reinterpret_cast<const uint32_t*>(&l);
}

__device__ __forceinline__ float2 cmulf(float2 a, float2 b) {
    return make_float2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}

// potential factor exp(-i tau V/hbar) on the pair (u, l) at column x of the row with
// coordinate y (the same product form of the standing wave as the CUDA-core x sweep:
// a_y = -2 s G cos(Theta), a_x = 4 eps s (y/w) G sin(Theta + zeta), applied as
// psi + (cos(theta) - 1) psi + i sin(theta)/|a| (alpha.a) psi)
__device__ __forceinline__ void potential(const SweepArgs& a, int pair, int x, float y, float y2,
                                          float st, float kap, float kap2, float e4, float2* u, float2* l) {
    const float4* xt = reinterpret_cast<const float4*>(a.xtab);
    const float4 t1 = __ldg(xt + a.nx + x);
    float ax = 0.0f, ay;
    if (a.kind == 1) {
        ay = -2.0f * st * t1.w;
    } else {
        const float4 t0 = __ldg(xt + x);
        const float G = t0.z * __expf(-y2 * t0.w);
        float th = t0.x - t0.y * y2;
        th -= 6.283185307f * rintf(th * 0.159154943f);
        float sn, cs;
        __sincosf(th, &sn, &cs);
        const float sg = st * G;
        ay = -2.0f * sg * cs;
        if (a.longitudinal) ax = e4 * sg * (y * t1.x) * (sn * t1.y + cs * t1.z);
    }
    const float a2 = ax * ax + ay * ay;
    const float th2 = kap2 * a2;
    float c1, s;
    if (th2 < 0.0625f) {
        c1 = th2 * (-0.5f + th2 * (1.0f / 24 + th2 * (-1.0f / 720 + th2 * (1.0f / 40320))));
        const float sinc = 1.0f + th2 * (-1.0f / 6 + th2 * (1.0f / 120 + th2 * (-1.0f / 5040 + th2 * (1.0f / 362880))));
        s = kap * sinc;
    } else {
        const float amag = sqrtf(a2);
        float sh, ch;
        sincosf(0.5f * kap * amag, &sh, &ch);
        c1 = -2.0f * sh * sh;
        s = 2.0f * sh * ch / amag;
    }
    const float sgp = pair == 0 ? 1.0f : -1.0f;
    const float2 q1 = make_float2(s * sgp * ay, s * ax), q2 = make_float2(-s * sgp * ay, s * ax);
    const float2 uu = *u, ll = *l;
    const float2 ql = cmulf(q1, ll), qu = cmulf(q2, uu);
    *u = make_float2(uu.x + (c1 * uu.x + ql.x), uu.y + (c1 * uu.y + ql.y));
    *l = make_float2(ll.x + (c1 * ll.x + qu.x), ll.y + (c1 * ll.y + qu.y));
}

// kinetic factor e^{i phi} [C - i S H0(pi)] / P at (kx, ky), from the same FP32 tables as the
// CUDA-core y sweep: psi/P + a psi - i b (H0/c) psi, then times 1 + f
__device__ __forceinline__ void kinetic(const SweepArgs& a, int pair, int kx, int ky, float2* u, float2* l) {
    const float2 ab = __ldg(reinterpret_cast<const float2*>(a.ktab) + (long long)ky * a.nx + kx);
    const float4 yv = __ldg(reinterpret_cast<const float4*>(a.kytab) + ky);
    const float pix = __ldg(reinterpret_cast<const float*>(a.kxtab) + kx);
    const float mc = a.mc_f, invP = a.invP_f;
    const float piy = pair == 0 ? yv.x : -yv.x;
    const float2 uu = *u, ll = *l;
    const float2 hu = make_float2(mc * uu.x + pix * ll.x + piy * ll.y, mc * uu.y + pix * ll.y - piy * ll.x);
    const float2 hl = make_float2(pix * uu.x - piy * uu.y - mc * ll.x, pix * uu.y + piy * uu.x - mc * ll.y);
    const float2 u1 = make_float2(uu.x * invP + (ab.x * uu.x + ab.y * hu.y), uu.y * invP + (ab.x * uu.y - ab.y * hu.x));
    const float2 l1 = make_float2(ll.x * invP + (ab.x * ll.x + ab.y * hl.y), ll.y * invP + (ab.x * ll.y - ab.y * hl.x));
    *u = make_float2(u1.x + (yv.y * u1.x - yv.z * u1.y), u1.y + (yv.y * u1.y + yv.z * u1.x));
    *l = make_float2(l1.x + (yv.y * l1.x - yv.z * l1.y), l1.y + (yv.y * l1.y + yv.z * l1.x));
}

// One full sweep (both FFTs and the pointwise factor) over lines of 1024 points.
// Persistent: each CTA loops over work items of 4 lines of one pair.
template <int AXIS>
__global__ void __launch_bounds__(THREADS, 2) tc_sweep(const SweepArgs a) {
    extern __shared__ __align__(128) unsigned char sm[];
    const int t = threadIdx.x, w = t >> 5;
    const uint32_t s0 = su32(sm);
    const uint32_t bar = s0 + OFF_BAR;
    uint32_t* slot = reinterpret_cast<uint32_t*>(sm + OFF_SLOT);
    // first FFT: inverse on the x axis, forward on the y axis; the second the other one
    constexpr int D1 = AXIS == AXIS_X ? +1 : -1;
    // B images: [inverse hi, inverse lo, forward hi, forward lo]
    const uint32_t b1 = s0 + OFF_B + (D1 > 0 ? 0u : 2u * BMAT), b2 = s0 + OFF_B + (D1 > 0 ? 2u * BMAT : 0u);

    // ---- setup: tensor memory, barrier, DFT matrices, this thread's twiddles
    if (w == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;"
                     :: "r"(s0 + OFF_SLOT), "r"(TMEM_COLS));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    if (t == 0) {
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" :: "r"(bar));
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    {
        const uint4* src = reinterpret_cast<const uint4*>(a.tc_b);
        uint4* dst = reinterpret_cast<uint4*>(sm + OFF_B);
        for (int i = t; i < (int)(4 * BMAT / 16); i += THREADS) dst[i] = __ldg(src + i);
    }
    // the thread's row r is its TMEM lane in every stage; half h of the CTA takes columns
    // [16 h, 16 h + 16) of it.  Row of (vector, line): x axis 32 line + vector (a warp's
    // lanes are consecutive points of one row: contiguous loads, conflict-free transposes),
    // y axis 4 vector + line (a warp spans 4 adjacent columns: 64-byte segments)
    auto rowof = [](int v, int l) { return AXIS == AXIS_X ? 32 * l + v : 4 * v + l; };
    const int r = t & 127, h = t >> 7;
    const int vec = AXIS == AXIS_X ? (r & 31) : (r >> 2), ln = AXIS == AXIS_X ? (r >> 5) : (r & 3);
    float2 tw[HALF];   // w_N^(D1 vec k) / 2^10, k in this half (the second FFT: conjugates)
    {
        const float2* tab = reinterpret_cast<const float2*>(a.tc_tw);
#pragma unroll
        for (int i = 0; i < HALF; ++i) {
            const int k = HALF * h + i;
            const float2 e = __ldg(tab + ((vec * k) & (N - 1)));
            tw[i] = make_float2(e.x * BSCALE_INV, (float)D1 * e.y * BSCALE_INV);
        }
    }
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t tmem = *slot;
    const uint32_t trow = tmem + ((uint32_t)((w & 3) * 32) << 16);   // this warp's lane quadrant

    // wait for the previous kernel in the stream (programmatic dependent launch)
    asm volatile("griddepcontrol.wait;" ::: "memory");
    const float sa = a.tc_scale[2 * AXIS], sb = a.tc_scale[2 * AXIS + 1];
    const float sop = sb * BSCALE_INV, sout = BSCALE_INV / (sa * sb);
    const int nx = a.nx, ny = a.ny;
    const int lines = AXIS == AXIS_X ? ny : nx;
    const int items = 2 * (lines / LC);
    const long long plane = (long long)nx * ny;
    const float4* in = reinterpret_cast<const float4*>(a.in);
    float4* out = reinterpret_cast<float4*>(a.out);
    uint32_t phase = 0;
    bool failed = false;

    // potential-step scalars (x axis)
    float st = 0.0f, ybase = 0.0f, kap = 0.0f, kap2 = 0.0f, e4 = 0.0f;
    if (AXIS == AXIS_X && a.op == OP_POTENTIAL && a.kind != 0) {
        const Clock ck = *a.clock;
        const StepScalars* ssp = a.steps + ((ck.step - ck.base) + a.n_local);
        st = ssp->s_f;
        ybase = ssp->ybase_f;
        kap = a.kappa_f;
        kap2 = kap * kap;
        e4 = a.eps4_f;
    }

    // one DFT stage: operands in shared memory -> D in TMEM, all threads wait for it
    auto stage = [&](uint32_t bmat) -> bool {
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
        __syncthreads();
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        // (a.tc_fault: test hook that issues nothing, so the bounded wait below runs out)
        if (t == 0 && !a.tc_fault) {
#pragma unroll
            for (int c = 0; c < 2; ++c) {
#pragma unroll
                for (int term = 0; term < 3; ++term) {
                    const uint32_t d = tmem + (uint32_t)(c * 64 + (term ? 128 : 0));
                    const uint32_t abase = s0 + (term == 1 ? OFF_ALO : OFF_AHI) + (uint32_t)c * TILE;
                    const uint32_t bbase = bmat + (term == 2 ? BMAT : 0u);
#pragma unroll
                    for (int ks = 0; ks < 4; ++ks)
                        mma_f16(d, sdesc(abase + (uint32_t)ks * 2 * LBO, LBO, SBO),
                                sdesc(bbase + (uint32_t)ks * 2 * BLBO, BLBO, BSBO), (term == 2 || ks) != 0);
                }
            }
            asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];"
                         :: "r"(bar) : "memory");
        }
        const bool ok = mbar_wait(bar, phase);
        phase ^= 1u;
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        // all threads agree before anyone touches TMEM or the operands again
        return __syncthreads_and(ok) != 0;
    };

    // 8 complex of both components of this thread's row, chunk j (columns 16 j ..):
    // large plus small accumulators
    auto read8 = [&](int j, float* vu, float* vl) {
        uint32_t bu[16], bl[16], su[16], sl[16];
        KD_TMEM_LD16(trow + 16 * j, bu);
        KD_TMEM_LD16(trow + 64 + 16 * j, bl);
        KD_TMEM_LD16(trow + 128 + 16 * j, su);
        KD_TMEM_LD16(trow + 192 + 16 * j, sl);
        tmem_wait2(bu, bl);
        tmem_wait2(su, sl);
#pragma unroll
        for (int i = 0; i < 16; ++i) {
            vu[i] = __uint_as_float(bu[i]) + __uint_as_float(su[i]);
            vl[i] = __uint_as_float(bl[i]) + __uint_as_float(sl[i]);
        }
    };
    // writes 4 consecutive complex of component c (hi and lo) into row r at column col
    auto put4 = [&](int c, int r, int col, const uint32_t* hi, const uint32_t* lo) {
        const uint32_t o = aoff(r, col) + (uint32_t)c * TILE;
        *reinterpret_cast<uint4*>(sm + OFF_AHI + o) = make_uint4(hi[0], hi[1], hi[2], hi[3]);
        *reinterpret_cast<uint4*>(sm + OFF_ALO + o) = make_uint4(lo[0], lo[1], lo[2], lo[3]);
    };
    auto put1 = [&](int c, int r, int col, uint32_t hi, uint32_t lo) {
        const uint32_t o = aoff(r, col) + (uint32_t)c * TILE;
        *reinterpret_cast<uint32_t*>(sm + OFF_AHI + o) = hi;
        *reinterpret_cast<uint32_t*>(sm + OFF_ALO + o) = lo;
    };
    // global float4 index of point n of line `line` in pair `pr`
    auto gidx = [&](int pr, int line, int n) -> long long {
        return AXIS == AXIS_X ? pr * plane + (long long)line * nx + n : pr * plane + (long long)n * nx + line;
    };

    for (int item = blockIdx.x; item < items && !failed; item += gridDim.x) {
        const int pr = item & 1;
        const int line = (item >> 1) * LC + ln;   // this thread's line
        // ---- load: row (vec, ln) of S1 holds x[vec + 32 q], q < 32, scaled by sa
#pragma unroll 2
        for (int j = 4 * h; j < 4 * h + 4; ++j) {
            uint32_t uh[4], ul[4], lh[4], ll[4];
#pragma unroll
            for (int i = 0; i < 4; ++i) {
                const float4 v = __ldcg(in + gidx(pr, line, vec + 32 * (4 * j + i)));
                split(v.x * sa, v.y * sa, &uh[i], &ul[i]);
                split(v.z * sa, v.w * sa, &lh[i], &ll[i]);
            }
            put4(0, r, 4 * j, uh, ul);
            put4(1, r, 4 * j, lh, ll);
        }
        // ---- S1, T1, transpose into S2 rows (k2, ln), column vec
        if (!stage(b1)) { failed = true; break; }
#pragma unroll
        for (int jj = 0; jj < 2; ++jj) {
            float du[16], dl[16];
            read8(2 * h + jj, du, dl);
#pragma unroll
            for (int k = 0; k < 8; ++k) {
                const int k2 = HALF * h + 8 * jj + k;
                const float2 yu = cmulf(make_float2(du[2 * k], du[2 * k + 1]), tw[8 * jj + k]);
                const float2 yl = cmulf(make_float2(dl[2 * k], dl[2 * k + 1]), tw[8 * jj + k]);
                uint32_t hw, lw;
                split(yu.x, yu.y, &hw, &lw);
                put1(0, rowof(k2, ln), vec, hw, lw);
                split(yl.x, yl.y, &hw, &lw);
                put1(1, rowof(k2, ln), vec, hw, lw);
            }
        }
        // ---- S2: row (k2 = vec, ln) now holds X[vec + 32 k1]; pointwise factor in place
        if (!stage(b1)) { failed = true; break; }
        {
            const float y = ybase + (float)line * a.dy_f;
            const float y2 = y * y;
#pragma unroll 1
            for (int j = 2 * h; j < 2 * h + 2; ++j) {
                float du[16], dl[16];
                read8(j, du, dl);
                uint32_t uh[4], ul[4], lh[4], ll[4];
#pragma unroll
                for (int k = 0; k < 8; ++k) {
                    const int k1 = 8 * j + k;
                    const int m = vec + 32 * k1;   // position along the line
                    float2 u = make_float2(du[2 * k], du[2 * k + 1]);
                    float2 l = make_float2(dl[2 * k], dl[2 * k + 1]);
                    if (AXIS == AXIS_X) {
                        if (a.op == OP_POTENTIAL && a.kind != 0) potential(a, pr, m, y, y2, st, kap, kap2, e4, &u, &l);
                    } else {
                        if (a.op == OP_KINETIC) kinetic(a, pr, line, m, &u, &l);
                    }
                    split(u.x * sop, u.y * sop, &uh[k & 3], &ul[k & 3]);
                    split(l.x * sop, l.y * sop, &lh[k & 3], &ll[k & 3]);
                    if ((k & 3) == 3) {
                        put4(0, r, k1 - 3, uh, ul);
                        put4(1, r, k1 - 3, lh, ll);
                    }
                }
            }
        }
        // ---- S3, T2 (conjugate twiddles), transpose into S4 rows (c2, ln), column vec
        if (!stage(b2)) { failed = true; break; }
#pragma unroll
        for (int jj = 0; jj < 2; ++jj) {
            float du[16], dl[16];
            read8(2 * h + jj, du, dl);
#pragma unroll
            for (int k = 0; k < 8; ++k) {
                const int c2 = HALF * h + 8 * jj + k;
                const float2 wc = make_float2(tw[8 * jj + k].x, -tw[8 * jj + k].y);
                const float2 yu = cmulf(make_float2(du[2 * k], du[2 * k + 1]), wc);
                const float2 yl = cmulf(make_float2(dl[2 * k], dl[2 * k + 1]), wc);
                uint32_t hw, lw;
                split(yu.x, yu.y, &hw, &lw);
                put1(0, rowof(c2, ln), vec, hw, lw);
                split(yl.x, yl.y, &hw, &lw);
                put1(1, rowof(c2, ln), vec, hw, lw);
            }
        }
        // ---- S4: row (c2 = vec, ln) holds Y[vec + 32 c1]; store
        if (!stage(b2)) { failed = true; break; }
#pragma unroll 1
        for (int j = 2 * h; j < 2 * h + 2; ++j) {
            float du[16], dl[16];
            read8(j, du, dl);
#pragma unroll
            for (int k = 0; k < 8; ++k) {
                const int c1 = 8 * j + k;
                const float4 v = make_float4(du[2 * k] * sout, du[2 * k + 1] * sout, dl[2 * k] * sout, dl[2 * k + 1] * sout);
                __stcg(out + gidx(pr, line, vec + 32 * c1), v);
            }
        }
        // the next item's loads overwrite the operands and its S1 the accumulators: every
        // thread must be done reading TMEM first
        asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
        __syncthreads();
    }
    if (failed) {
        if (t == 0) atomicOr(a.status, KD_STATUS_TC_TIMEOUT);
        // the products may still be running: wait (bounded) before freeing their memory
        mbar_wait(bar, phase ^ 1u);
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    if (w == 0)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" :: "r"(tmem), "r"(TMEM_COLS));
}

}  // namespace tc

bool tc_supported(int logn) { return logn == 10; }

cudaError_t launch_tc_sweep(int axis, const SweepArgs& a, cudaStream_t s) {
    static bool attr_done[2] = {false, false};
    static int nsm = 0;
    auto k = axis == AXIS_X ? tc::tc_sweep<AXIS_X> : tc::tc_sweep<AXIS_Y>;
    if (!attr_done[axis]) {
        cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, tc::SMEM);
        if (e != cudaSuccess) return e;
        attr_done[axis] = true;
    }
    if (nsm == 0) {
        int dev = 0;
        cudaError_t e = cudaGetDevice(&dev);
        if (e == cudaSuccess) e = cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
        if (e != cudaSuccess) return e;
    }
    const int lines = axis == AXIS_X ? a.ny : a.nx;
    const int items = 2 * (lines / tc::LC);
    const int grid = items < 2 * nsm ? items : 2 * nsm;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(grid);
    cfg.blockDim = dim3(tc::THREADS);
    cfg.dynamicSmemBytes = tc::SMEM;
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, k, a);
}

}  // namespace kd
