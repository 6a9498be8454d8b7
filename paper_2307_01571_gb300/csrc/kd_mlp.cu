// kd_mlp.cu -- the surrogate network: a fully connected MLP with exact-erf GELU hidden
// layers, trained on the batched solver's outputs (seeded parameter draws -> diffraction
// and spin-flip populations).  Hand-written kernels: tiled GEMM with fused bias / GELU
// epilogue (FP32 on the CUDA cores, or BF16 operands on the tcgen05 tensor cores with FP32
// accumulation in tensor memory), the GELU derivative, fixed-order column sums, MSE loss
// and Adam.  Every reduction runs in a fixed order, so training is bitwise reproducible.
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stdint.h>
#include <math.h>

#include <vector>

#include "../../include/kd.h"

namespace kd {
int set_error(int code, const char* msg);  // kd_api.cu
}

struct kd_mlp {
    int device = 0;
    int L = 0;                       // number of layers (weight matrices)
    std::vector<int> w;              // widths, L + 1 entries
    std::vector<size_t> woff, boff;  // parameter offsets of W_l [w[l+1]][w[l]] and b_l
    size_t nparam = 0;
    float* param = nullptr;          // all W and b
    float* grad = nullptr;
    float* m1 = nullptr;             // Adam moments
    float* m2 = nullptr;
    long long adam_t = 0;
    int cap = 0;                     // batch capacity of the activation buffers
    std::vector<float*> z;           // pre-activations per layer [cap][w[l+1]]
    std::vector<float*> a;           // activations per layer output [cap][w[l+1]] (a[0] = input)
    float* dbuf0 = nullptr;          // gradient ping-pong buffers [cap][max width]
    float* dbuf1 = nullptr;
    float* lossbuf = nullptr;        // [cap * w[L]] squared errors, then partials
    float* gx = nullptr;             // gathered minibatch inputs [cap][w[0]]
    float* gt = nullptr;             // gathered minibatch targets [cap][w[L]]
    int prec = 0;                    // KD_MLP_FP32 or KD_MLP_BF16 (tensor-core GEMMs)
    int* status = nullptr;           // set when a tensor-core GEMM's bounded wait gave up
};

namespace {

int err(int code, const char* msg) { return kd::set_error(code, msg); }

#define MLP_CUDA(call)                                                                   \
    do {                                                                                 \
        cudaError_t e_ = (call);                                                         \
        if (e_ != cudaSuccess) return err(e_ == cudaErrorMemoryAllocation ? KD_ERR_NOMEM : KD_ERR_CUDA, #call); \
    } while (0)

__device__ __forceinline__ float gelu(float x) { return 0.5f * x * (1.0f + erff(x * 0.70710678118654752f)); }
__device__ __forceinline__ float gelu_grad(float x) {
    return 0.5f * (1.0f + erff(x * 0.70710678118654752f)) + x * 0.39894228040143268f * expf(-0.5f * x * x);
}

// C[m][n] = sum_k A(m, k) B(k, n) (+ bias[n]; GELU) with A(m, k) = A[m sam + k sak] and
// B(k, n) = B[k sbk + n sbn].  64x64 tiles, 16-deep k slabs, 256 threads, 4x4 outputs
// per thread; the k loop runs in order (deterministic).  epi: 0 store, 1 bias, 2 bias
// then Z = C, Y = GELU(C).
__global__ void __launch_bounds__(256) k_gemm(const float* A, long sam, long sak, const float* B,
                                              long sbk, long sbn, float* C, float* Y, const float* bias,
                                              int M, int N, int K, int epi) {
    __shared__ float As[16][64 + 1];
    __shared__ float Bs[16][64 + 1];
    const int tx = threadIdx.x % 16, ty = threadIdx.x / 16;
    const int m0 = blockIdx.y * 64, n0 = blockIdx.x * 64;
    float acc[4][4] = {{0}};
    for (int k0 = 0; k0 < K; k0 += 16) {
        for (int e = threadIdx.x; e < 16 * 64; e += 256) {
            const int kk = e / 64, mm = e % 64;
            const int gm = m0 + mm, gk = k0 + kk;
            As[kk][mm] = (gm < M && gk < K) ? A[gm * sam + gk * sak] : 0.0f;
            const int gn = n0 + mm;
            Bs[kk][mm] = (gk < K && gn < N) ? B[gk * sbk + gn * sbn] : 0.0f;
        }
        __syncthreads();
#pragma unroll
        for (int kk = 0; kk < 16; ++kk) {
            float av[4], bv[4];
#pragma unroll
            for (int i = 0; i < 4; ++i) av[i] = As[kk][ty * 4 + i];
#pragma unroll
            for (int j = 0; j < 4; ++j) bv[j] = Bs[kk][tx * 4 + j];
#pragma unroll
            for (int i = 0; i < 4; ++i)
#pragma unroll
                for (int j = 0; j < 4; ++j) acc[i][j] = fmaf(av[i], bv[j], acc[i][j]);
        }
        __syncthreads();
    }
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const int m = m0 + ty * 4 + i, n = n0 + tx * 4 + j;
            if (m >= M || n >= N) continue;
            float v = acc[i][j];
            if (epi >= 1) v += bias[n];
            C[(long)m * N + n] = v;
            if (epi == 2) Y[(long)m * N + n] = gelu(v);
        }
}

// dZ = dY * GELU'(Z), elementwise
// ------------------------------------------------------ BF16 tensor-core GEMM -----
// The same product and epilogues as k_gemm with BF16 operands (rounded to nearest from
// the FP32 inputs while staging) on the 5th-generation tensor cores, FP32 accumulation in
// tensor memory.  One CTA of 128 threads computes a 128 x 32 tile of C (narrow tiles: the
// network's products are small, so more CTAs share them): thread r owns row m0 + r, which
// is TMEM lane r.  The k dimension runs in 64-deep slabs through two shared-memory stages
// in the no-swizzle K-major canonical layout (8-row x 16-byte core matrices: LBO = 128 B
// between core matrices along k, SBO = 1024 B between 8-row groups): while thread 0's four
// tcgen05.mma.kind::f16 (M 128, N 32, K 16; A and B both BF16) of slab j run, committed to
// the stage's mbarrier, the threads load slab j + 1 from global memory (16-byte loads where
// the operand is contiguous in k and aligned), wait for slab j - 1's products (bounded) and
// store into the stage those freed.  A wait that runs out sets *status, the CTA issues no
// further products, waits (bounded) for those in flight and skips the epilogue; the host
// reports KD_ERR_TIMEOUT.
namespace tcg {
constexpr int BN = 32;                                   // columns of C per CTA
constexpr uint32_t LBO = 128, SBO = 1024;
constexpr uint32_t A_BYTES = 16 * SBO, B_BYTES = (BN / 8) * SBO, STAGE = A_BYTES + B_BYTES;
constexpr uint32_t OFF_BAR = 2 * STAGE, OFF_SLOT = OFF_BAR + 16;
constexpr uint32_t SMEM = OFF_SLOT + 16;
constexpr uint32_t TMEM_COLS = 32;
// instruction descriptor (kind::f16): D FP32 (bits 4-5 = 1), A BF16 (bits 7-9 = 1), B BF16
// (bits 10-12 = 1), both K-major, N >> 3 at bit 17, M >> 4 at bit 24
constexpr uint32_t IDESC = (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(BN >> 3) << 17) |
                           ((uint32_t)(128 >> 4) << 24);
constexpr long long WAIT_LIMIT = 1ll << 20;

__device__ __forceinline__ uint32_t su32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }
__device__ __forceinline__ uint64_t sdesc(uint32_t saddr, uint32_t lbo, uint32_t sbo) {
    return (uint64_t)((saddr & 0x3FFFF) >> 4) | ((uint64_t)((lbo >> 4) & 0x3FFF) << 16) |
           ((uint64_t)((sbo >> 4) & 0x3FFF) << 32) | ((uint64_t)1 << 46);
}
__device__ __forceinline__ uint32_t pack_bf16(float lo, float hi) {
    const uint32_t a = (uint32_t)__bfloat16_as_ushort(__float2bfloat16_rn(lo));
    const uint32_t b = (uint32_t)__bfloat16_as_ushort(__float2bfloat16_rn(hi));
    return a | (b << 16);
}
__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t parity) {
    for (long long it = 0; it < WAIT_LIMIT; ++it) {
        uint32_t ok;
        asm volatile("{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
                     "selp.u32 %0, 1, 0, p;\n\t}" : "=r"(ok) : "r"(bar), "r"(parity) : "memory");
        if (ok) return true;
    }
    return false;
}
// eight consecutive k of one operand row (element (row, k) at p[row * sr + k * sk]), zero
// outside [0, K) or for rows out of range
__device__ __forceinline__ void load8(const float* p, long sr, long sk, int row, bool row_ok, int k, int K,
                                      float* v) {
    const float* q = p + (long)row * sr + (long)k * sk;
    if (row_ok && sk == 1 && k + 8 <= K && ((reinterpret_cast<uintptr_t>(q) & 15) == 0)) {
        const float4 a = __ldg(reinterpret_cast<const float4*>(q));
        const float4 b = __ldg(reinterpret_cast<const float4*>(q) + 1);
        v[0] = a.x; v[1] = a.y; v[2] = a.z; v[3] = a.w;
        v[4] = b.x; v[5] = b.y; v[6] = b.z; v[7] = b.w;
    } else {
#pragma unroll
        for (int e = 0; e < 8; ++e) v[e] = (row_ok && k + e < K) ? __ldg(q + (long)e * sk) : 0.0f;
    }
}
}  // namespace tcg

// one 64-deep slab of A (128 rows: 8 chunks of 8 k per thread) and B (32 rows n: thread t
// holds row t & 31, chunks 2 (t >> 5) and 2 (t >> 5) + 1) in registers
struct Slab {
    float a[8][8];
    float b[2][8];
};

__device__ __forceinline__ void slab_load(const float* A, long sam, long sak, const float* B, long sbk, long sbn,
                                          int m, int M, int n0, int N, int K, int k0, Slab& s) {
    const int t = threadIdx.x;
#pragma unroll
    for (int c = 0; c < 8; ++c) tcg::load8(A, sam, sak, m, m < M, k0 + 8 * c, K, s.a[c]);
    const int nn = t & 31, n = n0 + nn;
#pragma unroll
    for (int h = 0; h < 2; ++h) tcg::load8(B, sbn, sbk, n, n < N, k0 + 8 * (2 * (t >> 5) + h), K, s.b[h]);
}

__device__ __forceinline__ void slab_store(unsigned char* stage, const Slab& s) {
    const int t = threadIdx.x;
#pragma unroll
    for (int c = 0; c < 8; ++c) {
        const uint32_t o = (uint32_t)(t >> 3) * tcg::SBO + (uint32_t)c * tcg::LBO + (uint32_t)(t & 7) * 16;
        *reinterpret_cast<uint4*>(stage + o) =
            make_uint4(tcg::pack_bf16(s.a[c][0], s.a[c][1]), tcg::pack_bf16(s.a[c][2], s.a[c][3]),
                       tcg::pack_bf16(s.a[c][4], s.a[c][5]), tcg::pack_bf16(s.a[c][6], s.a[c][7]));
    }
    const int nn = t & 31;
#pragma unroll
    for (int h = 0; h < 2; ++h) {
        const int c = 2 * (t >> 5) + h;
        const uint32_t o = (uint32_t)(nn >> 3) * tcg::SBO + (uint32_t)c * tcg::LBO + (uint32_t)(nn & 7) * 16;
        *reinterpret_cast<uint4*>(stage + tcg::A_BYTES + o) =
            make_uint4(tcg::pack_bf16(s.b[h][0], s.b[h][1]), tcg::pack_bf16(s.b[h][2], s.b[h][3]),
                       tcg::pack_bf16(s.b[h][4], s.b[h][5]), tcg::pack_bf16(s.b[h][6], s.b[h][7]));
    }
}

__global__ void __launch_bounds__(128) k_gemm_bf16(const float* A, long sam, long sak, const float* B,
                                                   long sbk, long sbn, float* C, float* Y, const float* bias,
                                                   int M, int N, int K, int epi, int* status) {
    extern __shared__ __align__(1024) unsigned char sm[];
    const int t = threadIdx.x, w = t >> 5;
    const int m0 = blockIdx.y * 128, n0 = blockIdx.x * tcg::BN;
    const uint32_t s0 = tcg::su32(sm);
    const uint32_t bar[2] = {s0 + tcg::OFF_BAR, s0 + tcg::OFF_BAR + 8};
    if (w == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;"
                     :: "r"(s0 + tcg::OFF_SLOT), "r"(tcg::TMEM_COLS));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    if (t == 0) {
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" :: "r"(bar[0]));
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" :: "r"(bar[1]));
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t tmem = *reinterpret_cast<const uint32_t*>(sm + tcg::OFF_SLOT);
    const int m = m0 + t;
    const int nslab = (K + 63) / 64;
    uint32_t phase[2] = {0u, 0u};
    bool ok = true;
    int issued = 0;          // slabs whose products were issued (and committed)
    int waited = 0;          // slabs whose products were waited for
    Slab sl;
    if (nslab > 0) {
        slab_load(A, sam, sak, B, sbk, sbn, m, M, n0, N, K, 0, sl);
        slab_store(sm, sl);
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
        __syncthreads();
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    }
    for (int j = 0; j < nslab && ok; ++j) {
        const int b = j & 1;
        if (t == 0) {
            const uint32_t sa = s0 + (uint32_t)b * tcg::STAGE;
#pragma unroll
            for (int ks = 0; ks < 4; ++ks) {
                const uint64_t da = tcg::sdesc(sa + (uint32_t)ks * 2 * tcg::LBO, tcg::LBO, tcg::SBO);
                const uint64_t db = tcg::sdesc(sa + tcg::A_BYTES + (uint32_t)ks * 2 * tcg::LBO, tcg::LBO, tcg::SBO);
                const uint32_t acc = (j > 0 || ks > 0) ? 1u : 0u;
                asm volatile("{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
                             "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}"
                             :: "r"(tmem), "l"(da), "l"(db), "r"(tcg::IDESC), "r"(acc));
            }
            asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];"
                         :: "r"(bar[b]) : "memory");
        }
        issued = j + 1;
        // the next slab's global loads run while these products do
        if (j + 1 < nslab) slab_load(A, sam, sak, B, sbk, sbn, m, M, n0, N, K, 64 * (j + 1), sl);
        bool got = true;
        if (j >= 1) {   // slab j - 1's products read the stage slab j + 1 goes to
            got = tcg::mbar_wait(bar[b ^ 1], phase[b ^ 1]);
            if (got) {
                phase[b ^ 1] ^= 1u;
                waited = j;
            }
        }
        if (got && j + 1 < nslab) {
            slab_store(sm + (uint32_t)(b ^ 1) * tcg::STAGE, sl);
            asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        }
        asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
        ok = __syncthreads_and(got) != 0;
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    }
    // the last issued slab's products (and, after a failed wait, those still in flight:
    // each wait bounded, the first that runs out ends them)
    while (waited < issued) {
        const int b = waited & 1;
        if (!tcg::mbar_wait(bar[b], phase[b])) {
            ok = false;
            break;
        }
        phase[b] ^= 1u;
        ++waited;
    }
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    ok = __syncthreads_and(ok) != 0;
    if (ok && nslab > 0) {
        // row m's 32 columns from TMEM lane t: two 16-column loads
        const uint32_t trow = tmem + ((uint32_t)((w & 3) * 32) << 16);
        uint32_t r[32];
#pragma unroll
        for (int j = 0; j < 2; ++j)
            asm volatile("tcgen05.ld.sync.aligned.32x32b.x16.b32 "
                         "{%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
                         : "=r"(r[16 * j + 0]), "=r"(r[16 * j + 1]), "=r"(r[16 * j + 2]), "=r"(r[16 * j + 3]),
                           "=r"(r[16 * j + 4]), "=r"(r[16 * j + 5]), "=r"(r[16 * j + 6]), "=r"(r[16 * j + 7]),
                           "=r"(r[16 * j + 8]), "=r"(r[16 * j + 9]), "=r"(r[16 * j + 10]), "=r"(r[16 * j + 11]),
                           "=r"(r[16 * j + 12]), "=r"(r[16 * j + 13]), "=r"(r[16 * j + 14]), "=r"(r[16 * j + 15])
                         : "r"(trow + 16 * j));
        asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
        if (m < M) {
#pragma unroll
            for (int j = 0; j < tcg::BN; ++j) {
                const int n = n0 + j;
                if (n >= N) break;
                float c = __uint_as_float(r[j]);
                if (epi >= 1) c += bias[n];
                C[(long)m * N + n] = c;
                if (epi == 2) Y[(long)m * N + n] = gelu(c);
            }
        }
    }
    if (!ok && t == 0) atomicOr(status, 1);
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    if (w == 0)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" :: "r"(tmem), "r"(tcg::TMEM_COLS));
}

__global__ void k_gelu_back(const float* dY, const float* Z, float* dZ, long n) {
    for (long i = blockIdx.x * (long)blockDim.x + threadIdx.x; i < n; i += (long)gridDim.x * blockDim.x)
        dZ[i] = dY[i] * gelu_grad(Z[i]);
}

// db[n] = sum_m dZ[m][n], rows in order (one thread per column)
__global__ void k_colsum(const float* dZ, int M, int N, float* db) {
    const int n = blockIdx.x * blockDim.x + threadIdx.x;
    if (n >= N) return;
    float s = 0.0f;
    for (int m = 0; m < M; ++m) s += dZ[(long)m * N + n];
    db[n] = s;
}

// MSE over B x D outputs: dY = 2 (Y - T) / (B D), sq[i] = (Y - T)^2
__global__ void k_mse(const float* Y, const float* T, float* dY, float* sq, long n, float scale) {
    for (long i = blockIdx.x * (long)blockDim.x + threadIdx.x; i < n; i += (long)gridDim.x * blockDim.x) {
        const float d = Y[i] - T[i];
        dY[i] = scale * d;
        sq[i] = d * d;
    }
}

// fixed-order sum of n floats times scale into out[0] (one block)
__global__ void k_sum(const float* x, long n, float scale, float* out) {
    __shared__ double red[256];
    double s = 0.0;
    for (long i = threadIdx.x; i < n; i += blockDim.x) s += (double)x[i];
    red[threadIdx.x] = s;
    __syncthreads();
    for (int w = 128; w > 0; w >>= 1) {
        if ((int)threadIdx.x < w) red[threadIdx.x] += red[threadIdx.x + w];
        __syncthreads();
    }
    if (threadIdx.x == 0) out[0] = (float)(red[0] * scale);
}

// dst[i][:] = src[idx[i]][:] for i < n (rows of `width` floats); an index outside
// [0, nsrc) gives a row of zeros
__global__ void k_gather_rows(const float* src, int width, long nsrc, const int32_t* idx, int n, float* dst) {
    const long total = (long)n * width;
    for (long e = blockIdx.x * (long)blockDim.x + threadIdx.x; e < total; e += (long)gridDim.x * blockDim.x) {
        const int i = (int)(e / width), j = (int)(e % width);
        const long r = idx[i];
        dst[e] = (r >= 0 && r < nsrc) ? src[r * width + j] : 0.0f;
    }
}

__global__ void k_adam(float* p, const float* g, float* m1, float* m2, long n, float lr, float b1,
                       float b2, float eps, float c1, float c2) {
    for (long i = blockIdx.x * (long)blockDim.x + threadIdx.x; i < n; i += (long)gridDim.x * blockDim.x) {
        const float gi = g[i];
        const float a = b1 * m1[i] + (1.0f - b1) * gi;
        const float b = b2 * m2[i] + (1.0f - b2) * gi * gi;
        m1[i] = a;
        m2[i] = b;
        p[i] -= lr * (a / c1) / (sqrtf(b / c2) + eps);
    }
}

cudaError_t gemm(const kd_mlp* net, const float* A, long sam, long sak, const float* B, long sbk, long sbn,
                 float* C, float* Y, const float* bias, int M, int N, int K, int epi, cudaStream_t s) {
    if (net->prec == KD_MLP_BF16) {
        // two 20 KB stages: at most 5 CTAs per SM, whose tensor memory (32 columns each)
        // fits the SM's 512 columns, so no allocation waits
        static bool attr = false;
        constexpr int smem = (int)tcg::SMEM;
        if (!attr) {
            cudaError_t e = cudaFuncSetAttribute(k_gemm_bf16, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
            if (e != cudaSuccess) return e;
            attr = true;
        }
        dim3 grid((N + tcg::BN - 1) / tcg::BN, (M + 127) / 128);
        k_gemm_bf16<<<grid, 128, smem, s>>>(A, sam, sak, B, sbk, sbn, C, Y, bias, M, N, K, epi, net->status);
        return cudaGetLastError();
    }
    dim3 grid((N + 63) / 64, (M + 63) / 64);
    k_gemm<<<grid, 256, 0, s>>>(A, sam, sak, B, sbk, sbn, C, Y, bias, M, N, K, epi);
    return cudaGetLastError();
}

// KD_ERR_TIMEOUT (and the flag cleared) when a tensor-core GEMM's bounded wait gave up
// since the last check; synchronises the device
int check_status(kd_mlp* n) {
    int st = 0;
    MLP_CUDA(cudaMemcpy(&st, n->status, sizeof(int), cudaMemcpyDeviceToHost));
    if (!st) return KD_OK;
    MLP_CUDA(cudaMemset(n->status, 0, sizeof(int)));
    return err(KD_ERR_TIMEOUT, "kd_mlp: a tensor-core GEMM's wait for its products gave up");
}

int maxw(const kd_mlp* n) {
    int m = 0;
    for (int v : n->w) m = v > m ? v : m;
    return m;
}

int ensure_cap(kd_mlp* n, int batch) {
    if (batch <= n->cap) return KD_OK;
    for (float* p : n->z) cudaFree(p);
    for (size_t l = 1; l < n->a.size(); ++l) cudaFree(n->a[l]);
    cudaFree(n->dbuf0);
    cudaFree(n->dbuf1);
    cudaFree(n->lossbuf);
    cudaFree(n->gx);
    cudaFree(n->gt);
    n->gx = n->gt = nullptr;   // gathered-batch buffers, re-made at the new capacity
    n->z.assign(n->L, nullptr);
    n->a.assign(n->L + 1, nullptr);
    for (int l = 0; l < n->L; ++l) {
        MLP_CUDA(cudaMalloc(&n->z[l], sizeof(float) * (size_t)batch * n->w[l + 1]));
        MLP_CUDA(cudaMalloc(&n->a[l + 1], sizeof(float) * (size_t)batch * n->w[l + 1]));
    }
    MLP_CUDA(cudaMalloc(&n->dbuf0, sizeof(float) * (size_t)batch * maxw(n)));
    MLP_CUDA(cudaMalloc(&n->dbuf1, sizeof(float) * (size_t)batch * maxw(n)));
    MLP_CUDA(cudaMalloc(&n->lossbuf, sizeof(float) * ((size_t)batch * n->w[n->L] + 1)));
    n->cap = batch;
    return KD_OK;
}

// forward pass from device input x (batch rows): a[l+1] = act(a[l] W_l^T + b_l); the
// last layer is linear (its output is a[L])
int forward(kd_mlp* n, const float* x, int batch, cudaStream_t s) {
    n->a[0] = const_cast<float*>(x);
    for (int l = 0; l < n->L; ++l) {
        const int fi = n->w[l], fo = n->w[l + 1];
        const bool last = l == n->L - 1;
        float* out = last ? n->a[l + 1] : n->z[l];
        MLP_CUDA(gemm(n, n->a[l], fi, 1, n->param + n->woff[l], 1, fi, out, last ? nullptr : n->a[l + 1],
                      n->param + n->boff[l], batch, fo, fi, last ? 1 : 2, s));
    }
    return KD_OK;
}

// loss and gradients for targets t (device): returns via lossbuf[0] the mean squared error
int backward(kd_mlp* n, const float* t, int batch, cudaStream_t s) {
    const int D = n->w[n->L];
    const long nout = (long)batch * D;
    float* sq = n->lossbuf + 1;
    k_mse<<<(int)((nout + 255) / 256), 256, 0, s>>>(n->a[n->L], t, n->dbuf0, sq, nout, 2.0f / (float)nout);
    MLP_CUDA(cudaGetLastError());
    k_sum<<<1, 256, 0, s>>>(sq, nout, 1.0f / (float)nout, n->lossbuf);   // mean squared error
    MLP_CUDA(cudaGetLastError());
    float* dcur = n->dbuf0;   // gradient w.r.t. the output of layer l (pre-activation for the last)
    float* dnext = n->dbuf1;
    for (int l = n->L - 1; l >= 0; --l) {
        const int fi = n->w[l], fo = n->w[l + 1];
        if (l != n->L - 1) {   // through the GELU: dZ = dA * GELU'(Z)
            const long cnt = (long)batch * fo;
            k_gelu_back<<<(int)((cnt + 255) / 256), 256, 0, s>>>(dcur, n->z[l], dcur, cnt);
            MLP_CUDA(cudaGetLastError());
        }
        // dW_l[o][i] = sum_b dZ[b][o] a_l[b][i];  db_l[o] = sum_b dZ[b][o]
        MLP_CUDA(gemm(n, dcur, 1, fo, n->a[l], fi, 1, n->grad + n->woff[l], nullptr, nullptr, fo, fi, batch, 0, s));
        k_colsum<<<(fo + 127) / 128, 128, 0, s>>>(dcur, batch, fo, n->grad + n->boff[l]);
        MLP_CUDA(cudaGetLastError());
        if (l > 0) {  // dA_{l}[b][i] = sum_o dZ[b][o] W_l[o][i]
            MLP_CUDA(gemm(n, dcur, fo, 1, n->param + n->woff[l], fi, 1, dnext, nullptr, nullptr, batch, fi, fo, 0, s));
            float* tmp = dcur;
            dcur = dnext;
            dnext = tmp;
        }
    }
    return KD_OK;
}

int copy_io(void* dst, const void* src, size_t bytes, int32_t where_dst, int32_t where_src, cudaStream_t s) {
    cudaMemcpyKind k = where_src == KD_HOST ? (where_dst == KD_HOST ? cudaMemcpyHostToHost : cudaMemcpyHostToDevice)
                                            : (where_dst == KD_HOST ? cudaMemcpyDeviceToHost : cudaMemcpyDeviceToDevice);
    MLP_CUDA(cudaMemcpyAsync(dst, src, bytes, k, s));
    return KD_OK;
}

}  // namespace

extern "C" {

int kd_mlp_create(const int32_t* widths, int32_t nlayers, kd_mlp** out) {
    if (!widths || !out || nlayers < 1 || nlayers > 16) return err(KD_ERR_ARG, "kd_mlp_create: need 1..16 layers");
    for (int i = 0; i <= nlayers; ++i)
        if (widths[i] < 1 || widths[i] > 4096) return err(KD_ERR_ARG, "kd_mlp_create: widths must be in [1, 4096]");
    *out = nullptr;
    kd_mlp* n = new kd_mlp();
    if (cudaGetDevice(&n->device) != cudaSuccess) { delete n; return err(KD_ERR_CUDA, "kd_mlp_create: no CUDA device"); }
    n->L = nlayers;
    n->w.assign(widths, widths + nlayers + 1);
    size_t off = 0;
    for (int l = 0; l < nlayers; ++l) {
        n->woff.push_back(off);
        off += (size_t)n->w[l + 1] * n->w[l];
        n->boff.push_back(off);
        off += n->w[l + 1];
    }
    n->nparam = off;
    auto bail = [&](int rc) { kd_mlp_destroy(n); return rc; };
    if (cudaMalloc(&n->param, off * sizeof(float)) != cudaSuccess || cudaMalloc(&n->grad, off * sizeof(float)) != cudaSuccess ||
        cudaMalloc(&n->m1, off * sizeof(float)) != cudaSuccess || cudaMalloc(&n->m2, off * sizeof(float)) != cudaSuccess)
        return bail(err(KD_ERR_NOMEM, "kd_mlp_create: allocation failed"));
    if (cudaMalloc(&n->status, sizeof(int)) != cudaSuccess || cudaMemset(n->status, 0, sizeof(int)) != cudaSuccess)
        return bail(err(KD_ERR_NOMEM, "kd_mlp_create: allocation failed"));
    if (cudaMemset(n->param, 0, off * sizeof(float)) != cudaSuccess || cudaMemset(n->m1, 0, off * sizeof(float)) != cudaSuccess ||
        cudaMemset(n->m2, 0, off * sizeof(float)) != cudaSuccess || cudaMemset(n->grad, 0, off * sizeof(float)) != cudaSuccess)
        return bail(err(KD_ERR_CUDA, "kd_mlp_create: memset failed"));
    n->a.assign(nlayers + 1, nullptr);
    n->z.assign(nlayers, nullptr);
    *out = n;
    return KD_OK;
}

void kd_mlp_destroy(kd_mlp* n) {
    if (!n) return;
    cudaSetDevice(n->device);
    cudaDeviceSynchronize();
    for (float* p : n->z) cudaFree(p);
    for (size_t l = 1; l < n->a.size(); ++l) cudaFree(n->a[l]);
    cudaFree(n->dbuf0);
    cudaFree(n->dbuf1);
    cudaFree(n->lossbuf);
    cudaFree(n->gx);
    cudaFree(n->gt);
    cudaFree(n->status);
    cudaFree(n->param);
    cudaFree(n->grad);
    cudaFree(n->m1);
    cudaFree(n->m2);
    delete n;
}

int kd_mlp_num_params(kd_mlp* n, int64_t* count) {
    if (!n || !count) return err(KD_ERR_ARG, "kd_mlp_num_params: null argument");
    *count = (int64_t)n->nparam;
    return KD_OK;
}

int kd_mlp_set_params(kd_mlp* n, const float* p, int32_t where) {
    if (!n || !p) return err(KD_ERR_ARG, "kd_mlp_set_params: null argument");
    MLP_CUDA(cudaSetDevice(n->device));
    int rc = copy_io(n->param, p, n->nparam * sizeof(float), KD_DEVICE, where, 0);
    if (rc) return rc;
    MLP_CUDA(cudaMemset(n->m1, 0, n->nparam * sizeof(float)));
    MLP_CUDA(cudaMemset(n->m2, 0, n->nparam * sizeof(float)));
    n->adam_t = 0;
    MLP_CUDA(cudaDeviceSynchronize());
    return KD_OK;
}

int kd_mlp_get_params(kd_mlp* n, float* p, int32_t where) {
    if (!n || !p) return err(KD_ERR_ARG, "kd_mlp_get_params: null argument");
    MLP_CUDA(cudaSetDevice(n->device));
    int rc = copy_io(p, n->param, n->nparam * sizeof(float), where, KD_DEVICE, 0);
    if (rc) return rc;
    MLP_CUDA(cudaDeviceSynchronize());
    return check_status(n);
}

int kd_mlp_set_precision(kd_mlp* n, int32_t precision) {
    if (!n || (precision != KD_MLP_FP32 && precision != KD_MLP_BF16))
        return err(KD_ERR_ARG, "kd_mlp_set_precision: KD_MLP_FP32 or KD_MLP_BF16");
    n->prec = precision;
    return KD_OK;
}

int kd_mlp_forward(kd_mlp* n, const float* x, int32_t batch, float* y, int32_t where, void* cuda_stream) {
    if (!n || !x || !y || batch <= 0) return err(KD_ERR_ARG, "kd_mlp_forward: bad argument");
    MLP_CUDA(cudaSetDevice(n->device));
    cudaStream_t s = (cudaStream_t)cuda_stream;
    int rc = ensure_cap(n, batch);
    if (rc) return rc;
    const float* xd = x;
    if (where == KD_HOST) {
        rc = copy_io(n->dbuf1, x, sizeof(float) * (size_t)batch * n->w[0], KD_DEVICE, KD_HOST, s);
        if (rc) return rc;
        xd = n->dbuf1;
    }
    rc = forward(n, xd, batch, s);
    if (rc) return rc;
    rc = copy_io(y, n->a[n->L], sizeof(float) * (size_t)batch * n->w[n->L], where, KD_DEVICE, s);
    if (rc) return rc;
    if (where == KD_HOST) {
        MLP_CUDA(cudaStreamSynchronize(s));
        return check_status(n);
    }
    return KD_OK;
}

int kd_mlp_gradients(kd_mlp* n, const float* x, const float* t, int32_t batch, float* loss,
                     float* grads, int32_t where, void* cuda_stream) {
    if (!n || !x || !t || batch <= 0) return err(KD_ERR_ARG, "kd_mlp_gradients: bad argument");
    MLP_CUDA(cudaSetDevice(n->device));
    cudaStream_t s = (cudaStream_t)cuda_stream;
    int rc = ensure_cap(n, batch);
    if (rc) return rc;
    const float* xd = x;
    const float* td = t;
    float* tmp_x = nullptr;
    float* tmp_t = nullptr;
    if (where == KD_HOST) {  // staged through the gradient buffers' tail: copy to device scratch
        MLP_CUDA(cudaMalloc(&tmp_x, sizeof(float) * (size_t)batch * n->w[0]));
        MLP_CUDA(cudaMalloc(&tmp_t, sizeof(float) * (size_t)batch * n->w[n->L]));
        rc = copy_io(tmp_x, x, sizeof(float) * (size_t)batch * n->w[0], KD_DEVICE, KD_HOST, s);
        if (!rc) rc = copy_io(tmp_t, t, sizeof(float) * (size_t)batch * n->w[n->L], KD_DEVICE, KD_HOST, s);
        if (rc) { cudaFree(tmp_x); cudaFree(tmp_t); return rc; }
        xd = tmp_x;
        td = tmp_t;
    }
    rc = forward(n, xd, batch, s);
    if (!rc) rc = backward(n, td, batch, s);
    if (!rc && loss) rc = copy_io(loss, n->lossbuf, sizeof(float), where, KD_DEVICE, s);
    if (!rc && grads) rc = copy_io(grads, n->grad, n->nparam * sizeof(float), where, KD_DEVICE, s);
    if (where == KD_HOST) {
        cudaStreamSynchronize(s);
        if (!rc) rc = check_status(n);
    }
    cudaFree(tmp_x);
    cudaFree(tmp_t);
    return rc;
}

int kd_mlp_train_step_gather(kd_mlp* n, const float* x_all, const float* t_all, int64_t n_all,
                             const int32_t* idx, int32_t batch, float lr, float* loss_dev, void* cuda_stream) {
    if (!n || !x_all || !t_all || !idx || n_all <= 0 || batch <= 0 || !(lr > 0))
        return err(KD_ERR_ARG, "kd_mlp_train_step_gather: bad argument");
    MLP_CUDA(cudaSetDevice(n->device));
    cudaStream_t s = (cudaStream_t)cuda_stream;
    int rc = ensure_cap(n, batch);
    if (rc) return rc;
    if (!n->gx) {
        MLP_CUDA(cudaMalloc(&n->gx, (size_t)n->cap * n->w[0] * sizeof(float)));
        MLP_CUDA(cudaMalloc(&n->gt, (size_t)n->cap * n->w[n->L] * sizeof(float)));
    }
    const int win = n->w[0], wout = n->w[n->L];
    k_gather_rows<<<(batch * win + 255) / 256, 256, 0, s>>>(x_all, win, (long)n_all, idx, batch, n->gx);
    k_gather_rows<<<(batch * wout + 255) / 256, 256, 0, s>>>(t_all, wout, (long)n_all, idx, batch, n->gt);
    MLP_CUDA(cudaGetLastError());
    return kd_mlp_train_step(n, n->gx, n->gt, batch, lr, loss_dev, cuda_stream);
}

int kd_mlp_train_step(kd_mlp* n, const float* x, const float* t, int32_t batch, float lr,
                      float* loss_dev, void* cuda_stream) {
    if (!n || !x || !t || batch <= 0 || !(lr > 0)) return err(KD_ERR_ARG, "kd_mlp_train_step: bad argument");
    MLP_CUDA(cudaSetDevice(n->device));
    cudaStream_t s = (cudaStream_t)cuda_stream;
    int rc = ensure_cap(n, batch);
    if (rc) return rc;
    rc = forward(n, x, batch, s);
    if (!rc) rc = backward(n, t, batch, s);
    if (rc) return rc;
    ++n->adam_t;
    const float b1 = 0.9f, b2 = 0.999f;
    const float c1 = 1.0f - powf(b1, (float)n->adam_t), c2 = 1.0f - powf(b2, (float)n->adam_t);
    k_adam<<<(int)((n->nparam + 255) / 256), 256, 0, s>>>(n->param, n->grad, n->m1, n->m2, (long)n->nparam,
                                                          lr, b1, b2, 1e-8f, c1, c2);
    MLP_CUDA(cudaGetLastError());
    if (loss_dev) MLP_CUDA(cudaMemcpyAsync(loss_dev, n->lossbuf, sizeof(float), cudaMemcpyDeviceToDevice, s));
    return KD_OK;
}

}  // extern "C"
