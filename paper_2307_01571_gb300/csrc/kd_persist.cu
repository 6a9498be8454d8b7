// kd_persist.cu -- the persistent form of the batched step: the Strang steps of a chunk for
// every member of a batch (independent simulations on uneven grids, FP32) run in ONE
// kernel launch whose CTAs pull work items from a device queue.
//
// Work item = (step i of the chunk, sweep y or x, member m, group g): a CTA-full of the
// member's standalone launch blocks of that sweep (the fused y sweep with the kinetic
// factor, the merged x sweep with the potential factor, or on the chunk's last step the
// closing half x sweep), i.e. exactly the work the standalone kernels do, so a member
// advanced here equals the member advanced alone with the same launch variants, bit for
// bit.  Items are handed out in the order (i, sweep, m, g) by an atomic counter; an item
// waits until its member has completed every item of the previous sweep (per-member
// completion counters, acquire/release), the only dependency of a 2D FFT sweep.  Work is
// pulled only by running CTAs and every item depends on items handed out before it, so the
// queue always progresses without any co-residency assumption.  The waits are bounded: a
// clock64 budget, after which the CTA sets the launch's abort flag and the members' status
// (KD_STATUS_TC_TIMEOUT: "a bounded wait gave up"), and every CTA leaves the queue.
#include <cuda_runtime.h>

#include "kd_persist.h"
#include "kd_sweep.cuh"

namespace kd {

namespace {

constexpr int kThreads = 256;            // CTA size of the persistent kernel
// launch variants the kernel holds per axis: x radix-8 (default) and radix-4 Stockham
// stages; y the 256-thread radix-8 tiles of one pair (default) and the radix-4 tiles of
// both pairs, the latter up to 256 points (at 512 points it needs 512-thread CTAs)
constexpr int kVX0 = 0, kVX1 = 2, kVY0 = 3, kVY1 = 2;
constexpr int kMinLog = 4, kMaxLog = 9, kMaxLogVY1 = 8;

static_assert(sizeof(SweepArgs) % sizeof(int4) == 0, "SweepArgs copies as int4");

template <int LOGN, int AXIS, int VAR> struct Geo {
    static constexpr int V = VAR;
    using Cf = Cfg<float, LOGN, AXIS, V>;
    static constexpr int TH = Cf::THREADS;
    static constexpr int K = kThreads / TH;           // standalone blocks per CTA-full
    static constexpr int SMEM = K * Cf::SMEM_BYTES;
    static_assert(kThreads % TH == 0, "persistent CTA holds whole blocks");
};

// one item of one sweep instantiation; not inlined, so that register allocation is per
// instantiation (one function holding every path would spill).  Where K > 1 standalone
// blocks share the CTA, each synchronises on its own named barrier (1 + part; 0 is the
// CTA's, used between items), so the blocks do not wait for each other.
template <int LOGN, int AXIS, int SHAPE, int VAR>
__device__ __noinline__ void run_group(const SweepArgs& a, int g, unsigned char* smem, int nl) {
    using G = Geo<LOGN, AXIS, VAR>;
    using S = Sweep<float, LOGN, AXIS, SHAPE, G::V>;
    static_assert(G::K <= 15, "named barriers 1 .. 15");
    const int part = threadIdx.x / G::TH;
    S::template run_block<false>(a, g * G::K + part, threadIdx.x % G::TH, smem + part * G::Cf::SMEM_BYTES, nl,
                                 G::K > 1 ? 1 + part : 0);
}

template <int AXIS, int SHAPE, int VAR>
__device__ __forceinline__ void run_logn_v(int logn, const SweepArgs& a, int g, unsigned char* smem, int nl) {
    switch (logn) {
        case 4: run_group<4, AXIS, SHAPE, VAR>(a, g, smem, nl); break;
        case 5: run_group<5, AXIS, SHAPE, VAR>(a, g, smem, nl); break;
        case 6: run_group<6, AXIS, SHAPE, VAR>(a, g, smem, nl); break;
        case 7: run_group<7, AXIS, SHAPE, VAR>(a, g, smem, nl); break;
        case 8: run_group<8, AXIS, SHAPE, VAR>(a, g, smem, nl); break;
        default: run_group<9, AXIS, SHAPE, VAR>(a, g, smem, nl); break;
    }
}

// the second y variant, held up to kMaxLogVY1 (members of longer y axes never select it)
template <int SHAPE>
__device__ __forceinline__ void run_logn_y1(int logn, const SweepArgs& a, int g, unsigned char* smem, int nl) {
    switch (logn) {
        case 4: run_group<4, AXIS_Y, SHAPE, kVY1>(a, g, smem, nl); break;
        case 5: run_group<5, AXIS_Y, SHAPE, kVY1>(a, g, smem, nl); break;
        case 6: run_group<6, AXIS_Y, SHAPE, kVY1>(a, g, smem, nl); break;
        case 7: run_group<7, AXIS_Y, SHAPE, kVY1>(a, g, smem, nl); break;
        default: run_group<8, AXIS_Y, SHAPE, kVY1>(a, g, smem, nl); break;
    }
}

// alt selects the second variant of the axis
template <int AXIS, int SHAPE>
__device__ __forceinline__ void run_logn(int logn, int alt, const SweepArgs& a, int g, unsigned char* smem, int nl) {
    if constexpr (AXIS == AXIS_X) {
        if (alt) run_logn_v<AXIS, SHAPE, kVX1>(logn, a, g, smem, nl);
        else run_logn_v<AXIS, SHAPE, kVX0>(logn, a, g, smem, nl);
    } else {
        if (alt && logn <= kMaxLogVY1) run_logn_y1<SHAPE>(logn, a, g, smem, nl);
        else run_logn_v<AXIS, SHAPE, kVY0>(logn, a, g, smem, nl);
    }
}

__device__ __forceinline__ unsigned ld_acquire(const unsigned* p) {
    unsigned v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

// member index of item r (0 <= r < pre[n]) of a prefix-summed item count
__device__ __forceinline__ int find_member(const int* pre, int n, int r) {
    int lo = 0, hi = n - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (pre[mid] <= r) lo = mid; else hi = mid - 1;
    }
    return lo;
}

__global__ void __launch_bounds__(kThreads, 3) k_persist(const PersistPlan p) {
    extern __shared__ __align__(16) unsigned char smem[];
    // the current item, decoded by warp 0 (read by every thread after the item's barrier)
    __shared__ int s_go, s_item, s_m, s_g, s_i, s_ysweep, s_closing;
    // the item's sweep arguments, staged in shared memory (read many times by every thread)
    __shared__ __align__(16) SweepArgs s_args;
    const PersistMember* mem = p.members;
    const int S = p.items_per_step;
    const long long total = (long long)S * p.chunk;
    // thread 0 takes the next item from the queue while the CTA works on the current one
    int next_item = 0;
    if (threadIdx.x == 0) next_item = (int)atomicAdd(p.next, 1u);
    for (;;) {
        if (threadIdx.x < 32) {
            // warp 0: lane 0 takes the item, decodes it and waits for its dependency; the
            // warp stages its arguments; one CTA barrier then publishes all of it
            int go = 0, item = 0, m = 0, g = 0, i = 0, ysweep = 0, closing = 0;
            if (threadIdx.x == 0) {
                item = next_item;
                go = item < total && *(volatile const int*)p.abort == 0;
                if (go) {
                    next_item = (int)atomicAdd(p.next, 1u);
                    i = item / S;            // step of the chunk, 0-based
                    int r = item % S;
                    ysweep = r < p.y_items;
                    if (!ysweep) r -= p.y_items;
                    const int* pre = ysweep ? p.pre_y : p.pre_x;
                    m = find_member(pre, p.n, r);
                    g = r - pre[m];
                    closing = !ysweep && i + 1 == p.chunk && p.closing;
                    // dependency: every item of member m before this sweep
                    const PersistMember& M = mem[m];
                    const unsigned need = (unsigned)(i * (M.iy + M.ix) + (ysweep ? 0 : M.iy));
                    if (ld_acquire(p.done + m) < need) {
                        const long long t0 = clock64();
                        while (ld_acquire(p.done + m) < need) {
                            if (*(volatile const int*)p.abort) { go = 0; break; }
                            if (clock64() - t0 > p.budget_cycles) {
                                atomicExch(p.abort, 1);
                                atomicOr(M.status, KD_STATUS_TC_TIMEOUT);
                                go = 0;
                                break;
                            }
                            __nanosleep(128);
                        }
                    }
                }
            }
            const unsigned full = 0xffffffffu;
            go = __shfl_sync(full, go, 0);
            m = __shfl_sync(full, m, 0);
            ysweep = __shfl_sync(full, ysweep, 0);
            closing = __shfl_sync(full, closing, 0);
            if (go) {
                const PersistMember& M = mem[m];
                const int4* src = reinterpret_cast<const int4*>(ysweep ? &M.y : (closing ? &M.xc : &M.x));
                int4* dst = reinterpret_cast<int4*>(&s_args);
                for (int w = threadIdx.x; w < (int)(sizeof(SweepArgs) / sizeof(int4)); w += 32) dst[w] = src[w];
            }
            if (threadIdx.x == 0) {
                s_go = go;
                s_item = item;
                s_m = m;
                s_g = g;
                s_i = i;
                s_ysweep = ysweep;
                s_closing = closing;
            }
        }
        __syncthreads();
        if (!s_go) break;
        const int m = s_m, i = s_i, ysweep = s_ysweep, closing = s_closing;
        const PersistMember& M = mem[m];
        // the item's CTA-fulls of blocks, one after the other (a barrier between them, so
        // that no thread writes shared memory another still reads)
        const int per = ysweep ? M.gy : M.gx, nct = ysweep ? M.cy : M.cx;
        const int c0 = s_g * per, c1 = c0 + per < nct ? c0 + per : nct;
        for (int cf = c0; cf < c1; ++cf) {
            if (cf > c0) __syncthreads();
            if (ysweep) run_logn<AXIS_Y, SHAPE_F1F2>(M.ly, M.vy_alt, s_args, cf, smem, 0);
            else if (closing) run_logn<AXIS_X, SHAPE_F1>(M.lx, M.vx_alt, s_args, cf, smem, i + 1);
            else run_logn<AXIS_X, SHAPE_F1F2>(M.lx, M.vx_alt, s_args, cf, smem, i + 1);
        }
        __syncthreads();
        if (threadIdx.x == 0 && s_item != p.hold_item) {
            // release at GPU scope: the CTA's stores (ordered before this thread by the
            // barrier) are visible to whoever acquires the new count
            asm volatile("red.release.gpu.global.add.u32 [%0], %1;" ::"l"(p.done + m), "r"(1u) : "memory");
        }
    }
}

template <int LOGN, int AXIS, int VAR> void geo_v(int lines, int* ctas) {
    using G = Geo<LOGN, AXIS, VAR>;
    const int blocks = ((lines + G::Cf::BATCH - 1) / G::Cf::BATCH) * G::Cf::NPAIRS;
    *ctas = (blocks + G::K - 1) / G::K;
}
template <int LOGN> void geo_axis(int axis, int alt, int lines, int* ctas) {
    if (axis == AXIS_X) {
        if (alt) geo_v<LOGN, AXIS_X, kVX1>(lines, ctas); else geo_v<LOGN, AXIS_X, kVX0>(lines, ctas);
    } else {
        if constexpr (LOGN <= kMaxLogVY1) {
            if (alt) { geo_v<LOGN, AXIS_Y, kVY1>(lines, ctas); return; }
        }
        geo_v<LOGN, AXIS_Y, kVY0>(lines, ctas);
    }
}

template <int LOGN> int max_smem() {
    int y1 = 0;
    if constexpr (LOGN <= kMaxLogVY1) y1 = Geo<LOGN, AXIS_Y, kVY1>::SMEM;
    const int s[4] = {Geo<LOGN, AXIS_X, kVX0>::SMEM, Geo<LOGN, AXIS_X, kVX1>::SMEM,
                      Geo<LOGN, AXIS_Y, kVY0>::SMEM, y1};
    int m = 0;
    for (int v : s) m = v > m ? v : m;
    return m;
}

}  // namespace

bool persist_supported(int logn) { return logn >= kMinLog && logn <= kMaxLog; }

int persist_ctas(int axis, int alt, int logn, int lines) {
    int items = 0;
    switch (logn) {
        case 4: geo_axis<4>(axis, alt, lines, &items); break;
        case 5: geo_axis<5>(axis, alt, lines, &items); break;
        case 6: geo_axis<6>(axis, alt, lines, &items); break;
        case 7: geo_axis<7>(axis, alt, lines, &items); break;
        case 8: geo_axis<8>(axis, alt, lines, &items); break;
        case 9: geo_axis<9>(axis, alt, lines, &items); break;
        default: return -1;
    }
    return items;
}

int persist_variant_alt(int axis, int variant, int logn) {
    if (axis == AXIS_X) return variant == kVX1 ? 1 : 0;
    return variant == kVY1 && logn <= kMaxLogVY1 ? 1 : 0;
}

void persist_variants(int axis, int logn, int* v0, int* v1) {
    *v0 = axis == AXIS_X ? kVX0 : kVY0;
    *v1 = axis == AXIS_X ? kVX1 : (logn <= kMaxLogVY1 ? kVY1 : kVY0);
}

cudaError_t launch_persist(const PersistPlan& p, cudaStream_t s) {
    static int smem = 0, grid = 0;
    if (grid == 0) {
        int m = 0;
        const int sm[] = {max_smem<4>(), max_smem<5>(), max_smem<6>(), max_smem<7>(),
                          max_smem<8>(), max_smem<9>()};
        for (int v : sm) m = v > m ? v : m;
        cudaError_t e = cudaFuncSetAttribute(k_persist, cudaFuncAttributeMaxDynamicSharedMemorySize, m);
        if (e != cudaSuccess) return e;
        int per_sm = 0, dev = 0, sms = 0;
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_persist, kThreads, m);
        if (e != cudaSuccess) return e;
        e = cudaGetDevice(&dev);
        if (e != cudaSuccess) return e;
        e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        if (e != cudaSuccess) return e;
        if (per_sm < 1) return cudaErrorInvalidConfiguration;
        smem = m;
        grid = per_sm * sms;
    }
    k_persist<<<grid, kThreads, smem, s>>>(p);
    return cudaGetLastError();
}

}  // namespace kd
